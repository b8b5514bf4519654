"""The adjoint workload at full size: the 128^3 layered channel reservoir,
60 EREM steps, 16 observation cells, checkpoints every 10 steps.  The
gradient of the misfit with respect to ln K and T0 (the torch.autograd.Function
over the C ABI's adjoint) is checked against central finite differences of
the forward with h = 1e-4 on 8 random directions (the forward in FP64 with
its Leja schedules replayed and the spectral interval held, so that the
differences see the map the adjoint differentiates: a recomputed interval
alone moves the differences by a few 1e-5 here), and the FP32-bulk gradient
against the FP64 one.  The fields,
pressure scaling and capacities come from the oracle side.

ln K of this reservoir does not vary along x, so the head is linear in x and
every y and z face carries zero flux up to the rounding of the pressure
solve.  Upwinding has a kink at zero flux: a perturbation that varies along
x makes those fluxes O(h) of either sign, and central differences then
measure the mean of the two one-sided derivatives while the gradient is the
derivative of the computed map, whose sign at each such face is set by
rounding.  The ln K directions are therefore fields of (y, z), which leave the
head linear in x and the kinks uncrossed; the T0 directions are arbitrary.
General ln K directions are checked on random fields, whose fluxes are far
from zero, by the smaller adjoint tests."""
import numpy as np
import pytest

import cases as C
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    wl, obs, data = W.adjoint3d(128)
    case = C.from_workload(wl, pressure="cg")
    return E, case, obs, data, wl.steps


def _t(a, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _model(case, obs, data, steps, precision, replay=None, interval=None):
    import torch

    from paper_1209_5553_gb300.autograd import MisfitModel

    g = case.grid
    return MisfitModel(3, g.nx, g.ny, g.nz, case.gpu_physics(), _t(case.phi, torch.float64),
                       _t(case.lam, torch.float64), case.dt, steps, _t(obs, torch.int64),
                       _t(data, torch.float64), precision=precision, checkpoint=10, replay=replay,
                       interval=interval)


def _grads(case, obs, data, steps, precision):
    import torch

    from paper_1209_5553_gb300.autograd import misfit

    m = _model(case, obs, data, steps, precision)
    lnk = _t(case.lnk, torch.float64).requires_grad_(True)
    T0 = _t(case.T0, torch.float64).requires_grad_(True)
    L = misfit(lnk, T0, m)
    L.backward()
    out = (float(L.detach()), lnk.grad.cpu().numpy(), T0.grad.cpu().numpy(), list(m.schedules),
           m.interval)
    m.close()
    return out


@pytest.mark.timeout(1800)
def test_full_size_gradient_matches_central_differences(setup):
    import torch

    from paper_1209_5553_gb300.autograd import misfit

    E, case, obs, data, steps = setup
    L64, glnk64, gT064, sched, interval = _grads(case, obs, data, steps, "fp64")
    L32, glnk32, gT032, _, _ = _grads(case, obs, data, steps, "fp32_bulk")
    assert np.isfinite(glnk64).all() and np.isfinite(gT064).all()
    assert abs(L32 - L64) < 1e-6 * L64
    assert C.rel_l2(glnk32, glnk64) < 1e-3 and C.rel_l2(gT032, gT064) < 1e-3
    m = _model(case, obs, data, steps, "fp64", replay=sched, interval=interval)
    rng = np.random.default_rng(20120925 + 5)
    h = 1e-4
    with torch.no_grad():
        for _ in range(8):
            g = case.grid
            dk = np.repeat(rng.standard_normal(g.ny * g.nz), g.nx)
            dT = rng.standard_normal(case.n)
            Lp = float(misfit(_t(case.lnk + h * dk, torch.float64), _t(case.T0 + h * dT, torch.float64), m))
            Lm = float(misfit(_t(case.lnk - h * dk, torch.float64), _t(case.T0 - h * dT, torch.float64), m))
            fd = (Lp - Lm) / (2 * h)
            d64 = glnk64 @ dk + gT064 @ dT
            d32 = glnk32 @ dk + gT032 @ dT
            assert abs(fd - d64) < 1e-5 * max(abs(fd), 1e-3 * L64), (fd, d64)
            assert abs(fd - d32) < 1e-3 * max(abs(fd), 1e-3 * L64), (fd, d32)
    m.close()

"""Krylov phi_1 (§4.1) through the C ABI against the oracle.

FP64 (the Krylov path is FP64 in every context): the oracle replays the
substep lengths the GPU took and the results agree to 1e-11; the lengths
themselves must be the oracle's free-running ones (the step control is
FP64 arithmetic on the Arnoldi scalars, which differ from the oracle's by
rounding only).  Small grids where the Krylov dimension reaches N are exact;
on the 64^2 workload the Krylov and Leja paths agree to the tolerance."""
import numpy as np
import pytest

import cases as C
from oracle import krylov as K, leja, timestep as ts

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


@pytest.fixture(scope="module")
def E():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    return E


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _ctx(E, case, precision="fp64"):
    g = case.grid
    ctx = E.Context(g.dim, g.nx, g.ny, g.nz, physics=case.gpu_physics(), precision=precision)
    ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
    return ctx


CASES = {
    "heat2d_64": lambda: C.heat2d(64),
    "rect_37x23": lambda: C.heat2d_rect(37, 23),
    "channels3d_16": lambda: C.channels3d(16),
}


@pytest.mark.parametrize("name", list(CASES))
def test_phi1_apply_krylov_matches_oracle(E, name):
    case = CASES[name]()
    pb = case.problem()
    J, v = pb.J(case.T0), pb.G(case.T0)
    yinf = float(np.max(np.abs(case.T0)))
    free = K.phi1_krylov(J, v, case.dt, yinf)
    with _ctx(E, case) as ctx:
        out = _t(np.zeros(case.n))
        st = ctx.phi1_apply_krylov(_t(v), out)
        got = out.cpu().numpy()
    assert st.substeps == len(free.substeps) and st.substeps <= 64
    # later substeps start from states that differ by rounding, and r = J y + v
    # cancels: the lengths agree to about 1e-9 relative
    assert np.allclose(st.schedule, free.substeps, rtol=1e-7, atol=0)
    assert st.rejections == free.rejections
    rep = K.phi1_krylov(J, v, case.dt, yinf, K.KrylovOptions(replay=st.schedule))
    assert C.rel_l2(got, rep.value) < FP64_TOL


def _response(pb, T, dt, sched):
    """The oracle's own response to a rounding-size change of G (eps |J| |T|
    per cell, the size of the difference between two summation orders of the
    face fluxes), relative to T^{n+1}.  A step of few, long Krylov substeps
    combines basis vectors with large coefficients of both signs and can
    respond far above eps: on the 48^2 grid the second step responds with
    2e-10; on the 64^2 workload every step stays near 1e-13."""
    rng = np.random.default_rng(11)
    J, G = pb.J(T), pb.G(T)
    yinf = float(np.max(np.abs(T)))
    base = K.phi1_krylov(J, G, dt, yinf, K.KrylovOptions(replay=sched)).value
    scale = 2.0**-52 * (abs(J) @ np.abs(T))
    worst = 0.0
    for _ in range(3):
        Gp = G + scale * rng.standard_normal(G.size)
        alt = K.phi1_krylov(J, Gp, dt, yinf, K.KrylovOptions(replay=sched)).value
        worst = max(worst, C.rel_l2(T + alt, T + base))
    return worst


def test_erem_step_krylov_steps_match_oracle(E):
    # step by step the oracle replays the GPU's substeps; the bound is 1e-11
    # or, if larger, the sum over the steps so far of 20 times the oracle's
    # own response to rounding (which keeps it at 1e-11 on this workload)
    case = C.heat2d(64)
    pb = case.problem()
    T = case.T0.copy()
    bound = 0.0
    with _ctx(E, case) as ctx:
        Td = _t(case.T0)
        for step in range(4):
            st = ctx.erem_step_krylov(Td, case.dt)
            bound += 20.0 * _response(pb, T, case.dt, st.schedule)
            T, _ = ts.erem_step_krylov(pb, T, case.dt, K.KrylovOptions(replay=st.schedule))
            assert C.rel_l2(Td.cpu().numpy(), T) < max(FP64_TOL, bound), (step, bound)
    assert bound < FP64_TOL
    # against the Leja path over the same steps
    TL = case.T0.copy()
    for _ in range(4):
        TL, _ = ts.erem_step(pb, TL, case.dt)
    assert C.rel_l2(T, TL) < 1e-6


def test_krylov_is_exact_on_a_grid_smaller_than_the_basis(E):
    import scipy.linalg as sl

    case = C.heat2d_rect(3, 3)
    pb = case.problem()
    J, v = pb.J(case.T0).toarray(), pb.G(case.T0)
    n = v.size
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = case.dt * J
    A[:n, n] = v
    want = case.dt * sl.expm(A)[:n, n]
    with _ctx(E, case) as ctx:
        out = _t(np.zeros(n))
        st = ctx.phi1_apply_krylov(_t(v), out)
    assert st.substeps == 1 and st.dims[0] <= n
    assert C.rel_l2(out.cpu().numpy(), want) < 1e-12


def test_fp32_bulk_context_runs_krylov_in_fp64(E):
    case = C.heat2d(32)
    v = case.problem().G(case.T0)
    outs = []
    for prec in ("fp64", "fp32_bulk"):
        with _ctx(E, case, prec) as ctx:
            out = _t(np.zeros(case.n))
            ctx.phi1_apply_krylov(_t(v), out)
            outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_krylov_host_arrays_and_errors(E):
    case = C.heat2d(16)
    v = case.problem().G(case.T0)
    with _ctx(E, case) as ctx:
        host = np.zeros(case.n)
        ctx.phi1_apply_krylov(np.ascontiguousarray(v), host)
        dev = _t(np.zeros(case.n))
        ctx.phi1_apply_krylov(_t(v), dev)
        assert np.array_equal(host, dev.cpu().numpy())
        for bad in (E.krylov_opts(m=-1), E.krylov_opts(m=33), E.krylov_opts(tol=-1.0)):
            with pytest.raises(E.EremError) as ei:
                ctx.phi1_apply_krylov(_t(v), dev, bad)
            assert ei.value.status == E.EREM_EINVAL
        with pytest.raises(E.EremError) as ei:
            ctx.phi1_apply_krylov(_t(v), dev, E.krylov_opts(tol=1e-14, max_substeps=2))
        assert ei.value.status == E.EREM_ENOTCONV
    g = case.grid
    with E.Context(2, g.nx, g.ny, physics=case.gpu_physics()) as ctx:
        with pytest.raises(E.EremError) as ei:
            ctx.phi1_apply_krylov(_t(v), _t(np.zeros(case.n)))
        assert ei.value.status == E.EREM_EINVAL

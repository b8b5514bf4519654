"""Parity over the length of a timed run: 20 EREM steps of the 3D channel
reservoir at 64^3 (the 256^3 workload's family, dt = 1/32, tol 1e-6), FP64
with the oracle's schedules replayed and FP32-bulk free-running, against the
oracle's 20 steps on the same inputs.  The comparison is on the change the
run made, T^20 - T^0, as well as on the state."""
import numpy as np
import pytest

import cases as C
import workloads as W
from oracle import timestep as ts

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5
STEPS = 20


@pytest.fixture(scope="module")
def run():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    case = C.from_workload(W.channels3d(64), pressure="cg")
    prob = case.problem()
    T = case.T0.copy()
    states, scheds = [T], []
    for _ in range(STEPS):
        T, res = ts.erem_step(prob, T, case.dt)
        assert res.converged
        states.append(T)
        scheds.append(res.schedule)
    return E, case, states, scheds


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _gpu_run(E, case, precision, scheds=None):
    g = case.grid
    out, got_s = [], []
    with E.Context(3, g.nx, g.ny, g.nz, physics=case.gpu_physics(), precision=precision) as ctx:
        T = _t(case.T0)
        ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        for k in range(STEPS):
            opts = E.leja_opts(replay=scheds[k]) if scheds else None
            got_s.append(ctx.erem_step(T, case.dt, opts=opts).schedule)
            out.append(T.cpu().numpy())
    return out, got_s


@pytest.mark.timeout(1200)
def test_twenty_steps_fp64_replayed(run):
    E, case, states, scheds = run
    out, got_s = _gpu_run(E, case, "fp64", scheds)
    assert got_s == scheds
    for k in (0, 9, STEPS - 1):
        assert C.rel_l2(out[k], states[k + 1]) < FP64_TOL, k
        assert C.rel_l2(out[k] - case.T0, states[k + 1] - case.T0) < 10 * FP64_TOL, k


@pytest.mark.timeout(1200)
def test_twenty_steps_fp32_bulk_free_running(run):
    E, case, states, scheds = run
    out, got_s = _gpu_run(E, case, "fp32_bulk")
    for k in (0, 9, STEPS - 1):
        assert C.rel_l2(out[k], states[k + 1]) < FP32_TOL, k
        assert C.rel_l2(out[k] - case.T0, states[k + 1] - case.T0) < FP32_TOL, k
    # a free-running stop may legitimately move by a term or two
    assert all(g[0] == s[0] and max(abs(a - b) for a, b in zip(g[1:], s[1:])) <= 2
               for g, s in zip(got_s, scheds))

"""Parity at the size and launch configuration bench.py times: the 256^3
layered reservoir with channels (16.8 M cells, dt = 1/32, tol 1e-6), one
EREM step through the C ABI against the CPU oracle on the same inputs, and
EREM's exactness on this linear problem (one step of 2 dt equals two steps
of dt), a property that holds at any size.  The oracle step takes about a
minute on the host."""
import numpy as np
import pytest

import cases as C
import workloads as W
from oracle import timestep as ts

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def full():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    case = C.from_workload(W.channels3d(256), pressure="cg")
    T1, res = ts.erem_step(case.problem(), case.T0, case.dt)
    return E, case, T1, res


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _step(E, case, precision, steps, dt, opts=None):
    g = case.grid
    with E.Context(3, g.nx, g.ny, g.nz, physics=case.gpu_physics(), precision=precision) as ctx:
        T = _t(case.T0)
        ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), dt)
        scheds = []
        for _ in range(steps):
            scheds.append(ctx.erem_step(T, dt, opts=opts).schedule)
        return T.cpu().numpy(), scheds


@pytest.mark.timeout(1800)
def test_full_size_step_fp64_matches_oracle(full):
    E, case, T1, res = full
    got, scheds = _step(E, case, "fp64", 1, case.dt, E.leja_opts(replay=res.schedule))
    assert scheds[0] == res.schedule
    assert C.rel_l2(got, T1) < FP64_TOL
    assert C.rel_l2(got - case.T0, T1 - case.T0) < 1e-10


@pytest.mark.timeout(1800)
def test_full_size_step_fp32_bulk_matches_oracle(full):
    # the 1e-5 bound holds for the increment T^{n+1} - T^n the step computes,
    # not only for the state (whose background temperature dominates its norm)
    E, case, T1, res = full
    got, scheds = _step(E, case, "fp32_bulk", 1, case.dt)
    assert C.rel_l2(got, T1) < FP32_TOL
    assert C.rel_l2(got - case.T0, T1 - case.T0) < FP32_TOL
    assert abs(scheds[0][1] - res.degrees[0]) <= 2
    # with the oracle's schedule replayed the difference is FP32 rounding alone
    rep, scheds = _step(E, case, "fp32_bulk", 1, case.dt, E.leja_opts(replay=res.schedule))
    assert scheds[0] == res.schedule
    assert C.rel_l2(rep - case.T0, T1 - case.T0) < FP32_TOL


@pytest.mark.timeout(1800)
def test_full_size_exactness_on_the_linear_problem(full):
    E, case, _, _ = full
    opts = E.leja_opts(tol=1e-10)
    one, _ = _step(E, case, "fp64", 1, 2 * case.dt, opts)
    two, _ = _step(E, case, "fp64", 2, case.dt, opts)
    assert C.rel_l2(one - case.T0, two - case.T0) < 1e-7


@pytest.mark.timeout(1800)
def test_full_size_fast_leja_step_matches_oracle(full):
    # the fast (midpoint-candidate) Leja points at 256^3, FP64, the oracle's
    # schedule with the same points replayed
    from oracle.leja import LejaOptions

    E, case, _, _ = full
    T1, res = ts.erem_step(case.problem(), case.T0, case.dt, LejaOptions(points="fast"))
    g = case.grid
    with E.Context(3, g.nx, g.ny, g.nz, physics=case.gpu_physics(), precision="fp64") as ctx:
        ctx.set_leja_points("fast")
        T = _t(case.T0)
        ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        st = ctx.erem_step(T, case.dt, opts=E.leja_opts(replay=res.schedule))
        got = T.cpu().numpy()
    assert st.schedule == res.schedule
    assert C.rel_l2(got, T1) < FP64_TOL


@pytest.mark.timeout(1800)
def test_full_size_forced_step_matches_oracle(full):
    # the non-autonomous step (eq. nEERMg) at 256^3 with a time-dependent
    # inflow temperature: FP64 with the oracle's [s, m.., m_phi2] replayed,
    # FP32-bulk free-running
    from oracle import nonauto as NA

    E, case, _, _ = full
    T_in, rate = 70.0, 40.0
    T1, res = NA.erem_step_forced(case.problem(), case.T0, case.dt, T_in, rate)
    g = case.grid
    for prec, tol, opts in (("fp64", FP64_TOL, E.leja_opts(replay=res.schedule)), ("fp32_bulk", FP32_TOL, None)):
        with E.Context(3, g.nx, g.ny, g.nz, physics=case.gpu_physics(), precision=prec) as ctx:
            T = _t(case.T0)
            ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
            ctx.erem_step_forced(T, case.dt, T_in, rate, opts=opts)
            got = T.cpu().numpy()
        assert C.rel_l2(got, T1) < tol, prec
        inc_tol = 10 * tol if prec == "fp64" else tol
        assert C.rel_l2(got - case.T0, T1 - case.T0) < inc_tol, prec

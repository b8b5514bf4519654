"""Non-autonomous EREM (eq. ``nEERMg``) through the C ABI against the oracle
(oracle/nonauto.py): a time-dependent inflow temperature T_in(t) = 60 +
20 sin(8 t), FP64 with the oracle's schedules [s, m_1..m_s, m_phi2]
replayed (1e-11) and free-running on the oracle's own schedule, FP32-bulk
(1e-5), forced substeps, the autonomous limit and the argument errors."""
import math

import numpy as np
import pytest

import cases as C
from oracle import nonauto as NA
from oracle.leja import LejaOptions

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def E():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    return E


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _ctx(E, case, precision):
    d, nx, ny, nz = case.dims()
    g = case.grid
    return E.Context(d, nx, ny, nz, physics=case.gpu_physics(), precision=precision,
                     lx=g.lx, ly=g.ly, lz=g.lz)


def tin(t):
    return 60.0 + 20.0 * math.sin(8.0 * t)


def rate(t):
    return 160.0 * math.cos(8.0 * t)


def _oracle(case, steps, opts=None):
    pb = case.problem(case.T0)
    T = case.T0.copy()
    scheds = []
    for k in range(steps):
        t = k * case.dt
        o = opts(k) if callable(opts) else opts
        T, res = NA.erem_step_forced(pb, T, case.dt, tin(t), rate(t), o)
        assert res.converged
        scheds.append(res.schedule)
    return T, scheds


CASES = [("heat2d_64", lambda: C.heat2d(64)),
         ("ragged_37x23", lambda: C.heat2d_rect(37, 23)),
         ("box_12x10x7", lambda: C.random_case(3, 12, 10, 7, seed=5))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_forced_steps_match_oracle(E, name, make):
    case = make()
    steps = 4
    T_ref, scheds = _oracle(case, steps)
    fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
    for prec, tol in (("fp64", FP64_TOL), ("fp32_bulk", FP32_TOL)):
        for replay in ((True, False) if prec == "fp64" else (False,)):
            with _ctx(E, case, prec) as ctx:
                T = _t(case.T0)
                got_s = []
                for k in range(steps):
                    t = k * case.dt
                    opts = E.leja_opts(replay=scheds[k]) if replay else None
                    st = ctx.erem_step_forced(T, case.dt, tin(t), rate(t),
                                              *(fields if k == 0 else (None,) * 4), opts=opts)
                    got_s.append(st.schedule_forced)
                got = T.cpu().numpy()
            assert C.rel_l2(got, T_ref) < tol, (prec, replay)
            assert C.rel_l2(got - case.T0, T_ref - case.T0) < 1e3 * tol
            if prec == "fp64":
                assert got_s == scheds, (got_s, scheds)


@pytest.mark.parametrize("s", [2, 4])
def test_forced_substeps_match_oracle(E, s):
    # s pieces: the substep right-hand sides carry k delta D_t G and every
    # piece adds the same phi_2 increment
    case = C.heat2d_rect(24, 20)
    sched = [s] + [30] * s + [25]
    T_ref, _ = _oracle(case, 2, LejaOptions(replay=sched))
    with _ctx(E, case, "fp64") as ctx:
        T = _t(case.T0)
        for k in range(2):
            fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
            st = ctx.erem_step_forced(T, case.dt, tin(k * case.dt), rate(k * case.dt), *fields,
                                      opts=E.leja_opts(replay=sched))
            assert st.schedule_forced == sched
        got = T.cpu().numpy()
    assert C.rel_l2(got, T_ref) < FP64_TOL


def test_constant_inflow_is_the_autonomous_step(E):
    case = C.heat2d(32)
    fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
    with _ctx(E, case, "fp64") as ctx:
        T1 = _t(case.T0)
        s1 = ctx.erem_step_forced(T1, case.dt, case.phys.T_inflow, 0.0, *fields)
        T2 = _t(case.T0)
        s2 = ctx.erem_step(T2, case.dt, *fields)
    assert s1.schedule == s2.schedule and s1.degree_phi2 == 1
    a, b = T1.cpu().numpy(), T2.cpu().numpy()
    assert C.rel_l2(a - case.T0, b - case.T0) < 1e-13


def test_forced_step_errors(E):
    case = C.heat2d(16)
    fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
    with _ctx(E, case, "fp64") as ctx:
        T = _t(case.T0)
        for bad in ([1, 5], [2, 5, 5], [1, 5, 0]):
            with pytest.raises(E.EremError) as ei:
                ctx.erem_step_forced(T, case.dt, 60.0, 1.0, *fields, opts=E.leja_opts(replay=bad))
            assert ei.value.status == E.EREM_EINVAL
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step_forced(T, case.dt, float("nan"), 1.0, *fields)
        assert ei.value.status == E.EREM_EINVAL
        assert np.array_equal(T.cpu().numpy(), case.T0)
    nl = C.random_case(2, 10, 8, seed=7, fluid_model=1)
    with _ctx(E, nl, "fp64") as ctx:
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step_forced(_t(nl.T0), nl.dt, 60.0, 1.0, _t(nl.p), _t(nl.lnk), _t(nl.phi),
                                 _t(nl.lam))
        assert ei.value.status == E.EREM_EINVAL

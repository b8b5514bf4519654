"""Sequential (Trotter) coupling of §3.2 on the GPU: per step the steady
pressure at T^n, the Darcy fluxes with the viscosity at T^n, then one EREM
heat step with the T-dependent fluid laws (the 1024^2 workload's physics at
24 x 24 cells), against the oracle's sequential_step."""
import numpy as np
import pytest

import cases as C
import workloads as W
from oracle import fv, timestep as ts

pytestmark = pytest.mark.gpu

STEPS = 3
CG_TOL = 1e-13


def _setup():
    wl = W.coupled2d(n=24, steps=STEPS, dt=0.005)
    g = fv.Grid(2, 24, 24)
    base = fv.Physics(head_left=1.0, head_right=0.0, T_inflow=80.0, fluid_model=1)
    p0 = ts.pressure_solve_direct(g, base, wl.lnk, wl.T0)
    U = fv.darcy_fluxes(g, base, wl.lnk, p0, wl.T0)[0][:, :, 0].sum()
    rc = W.rhoc_for_peclet(50.0, 2.0, U)
    ph = fv.Physics(rc, rc, 1.0, 0.0, 80.0, 1)
    T = wl.T0.copy()
    ps, scheds, Ts = [], [], [T.copy()]
    for _ in range(STEPS):
        T, p, res = ts.sequential_step(g, ph, wl.lnk, wl.phi, wl.lam, T, None, wl.dt)
        ps.append(p)
        scheds.append(res.schedule)
        Ts.append(T.copy())
    return wl, g, ph, ps, scheds, Ts


@pytest.fixture(scope="module")
def setup():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    return (E,) + _setup()


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_coupled_steps_with_oracle_pressure(setup):
    E, wl, g, ph, ps, scheds, Ts = setup
    with E.Context(2, 24, 24, physics=E.Physics(ph.rhoc_f, ph.rhoc_s, 1.0, 0.0, 80.0, 1)) as ctx:
        T = _t(wl.T0)
        for k in range(STEPS):
            ctx.erem_step(T, wl.dt, _t(ps[k]), _t(wl.lnk), _t(wl.phi), _t(wl.lam),
                          opts=E.leja_opts(replay=scheds[k]))
        got = T.cpu().numpy()
    assert C.rel_l2(got, Ts[-1]) < 1e-11


def test_coupled_steps_with_gpu_pressure_in_the_loop(setup):
    E, wl, g, ph, ps, scheds, Ts = setup
    # pressure error bound of a CG stopped at CG_TOL (see test_gpu_solvers.py),
    # largest over the steps; T inherits it through the fluxes at most linearly
    bound = 0.0
    for k in range(STEPS):
        A, b = fv.pressure_system(g, ph, wl.lnk, Ts[k])
        smin = np.linalg.svd(A.toarray(), compute_uv=False).min()
        bound = max(bound, 10 * CG_TOL * np.linalg.norm(b) / smin / np.linalg.norm(ps[k]))
    with E.Context(2, 24, 24, physics=E.Physics(ph.rhoc_f, ph.rhoc_s, 1.0, 0.0, 80.0, 1)) as ctx:
        T = _t(wl.T0)
        p = _t(fv.linear_head_guess(g, ph))
        for k in range(STEPS):
            ctx.pressure_solve(_t(wl.lnk), T, p, tol=CG_TOL, maxit=20000)
            ctx.erem_step(T, wl.dt, p, _t(wl.lnk), _t(wl.phi), _t(wl.lam),
                          opts=E.leja_opts(replay=scheds[k]))
        got = T.cpu().numpy()
    inc = np.linalg.norm(Ts[-1] - wl.T0) / np.linalg.norm(Ts[-1])
    assert C.rel_l2(got, Ts[-1]) < max(1e-11, 10 * STEPS * bound * inc), bound


def test_coupled_step_trotter_and_strang_match_oracle(setup):
    # the C ABI's coupled_step: Trotter against the oracle's sequential
    # steps, Strang (heat dt/2, pressure, heat dt/2) against strang_step,
    # each heat step replaying the oracle's schedule; the pressure CG error
    # enters through the fluxes (bound as above)
    import torch

    E, wl, g, ph, ps, scheds, Ts = setup
    phys = E.Physics(ph.rhoc_f, ph.rhoc_s, 1.0, 0.0, 80.0, 1)
    T_s = wl.T0.copy()
    p_s = ts.pressure_solve_direct(g, ph, wl.lnk, T_s)
    Tp_s = T_s
    s_scheds, s_T, bound = [], [], 0.0
    for _ in range(STEPS):
        T_s, p_s, Tp_s, (r1, r2) = ts.strang_step(g, ph, wl.lnk, wl.phi, wl.lam, T_s, p_s, wl.dt,
                                                  T_p=Tp_s)
        s_scheds.append((r1.schedule, r2.schedule))
        A, b = fv.pressure_system(g, ph, wl.lnk, T_s)
        smin = np.linalg.svd(A.toarray(), compute_uv=False).min()
        bound = max(bound, 10 * CG_TOL * np.linalg.norm(b) / smin / np.linalg.norm(p_s))
    s_T = T_s
    fields = (_t(wl.lnk), _t(wl.phi), _t(wl.lam))
    with E.Context(2, 24, 24, physics=phys) as ctx:
        T = _t(wl.T0)
        p = _t(fv.linear_head_guess(g, ph))
        T_p = torch.empty_like(T)
        for k in range(STEPS):
            st, pst = ctx.coupled_step(T, p, *fields, wl.dt, E.EREM_SPLIT_TROTTER, pressure_tol=CG_TOL,
                                       opts=[E.leja_opts(replay=scheds[k])], T_p=T_p)
            assert pst.lin_resid <= CG_TOL and st[0].schedule == scheds[k]
        got_trotter = T.cpu().numpy()
        got_Tp_trotter = T_p.cpu().numpy()   # T^n of the last step: its pressure's temperature
        T = _t(wl.T0)
        p = _t(fv.linear_head_guess(g, ph))
        ctx.pressure_solve(fields[0], T, p, tol=CG_TOL)
        T_p = T.clone()                  # the pressure was solved at T^0
        for k in range(STEPS):
            st, pst = ctx.coupled_step(T, p, *fields, wl.dt, E.EREM_SPLIT_STRANG, pressure_tol=CG_TOL,
                                       opts=[E.leja_opts(replay=s) for s in s_scheds[k]], T_p=T_p)
            assert [s.schedule for s in st] == list(s_scheds[k])
        got_strang = T.cpu().numpy()
        got_Tp = T_p.cpu().numpy()
        p_got = p.cpu().numpy()
        with pytest.raises(ValueError):
            ctx.coupled_step(T, p, *fields, wl.dt, E.EREM_SPLIT_STRANG, opts=[E.leja_opts()])
        with pytest.raises(E.EremError) as ei:
            ctx.coupled_step(T, p, *fields, wl.dt, 7)
        assert ei.value.status == E.EREM_EINVAL
        with pytest.raises(E.EremError) as ei:   # T_p must not alias T
            ctx.coupled_step(T, p, *fields, wl.dt, E.EREM_SPLIT_STRANG, T_p=T)
        assert ei.value.status == E.EREM_EINVAL
    inc = np.linalg.norm(Ts[-1] - wl.T0) / np.linalg.norm(Ts[-1])
    assert C.rel_l2(got_trotter, Ts[-1]) < max(1e-11, 10 * STEPS * bound * inc)
    assert C.rel_l2(got_strang, s_T) < max(1e-11, 10 * STEPS * bound * inc)
    assert C.rel_l2(got_Tp, Tp_s) < max(1e-11, 10 * STEPS * bound * inc)
    assert C.rel_l2(got_Tp_trotter, Ts[-2]) < max(1e-11, 10 * STEPS * bound * inc)
    assert C.rel_l2(p_got, p_s) < 10 * bound
    # the two splittings differ at the splitting error, far above the bound
    assert C.rel_l2(got_strang, got_trotter) > 1e3 * max(1e-11, 10 * STEPS * bound * inc)

"""Parity at the size bench.py times for the coupled workload: the 1024^2
sequential pressure/temperature steps with the T-dependent fluid laws (§3.2,
sequential approach), two steps against the oracle's sequential_step
(pressure by a sparse direct solve), and one ROS2(1) step (eq. ROSMh, Table
ros2) against the oracle's ros2_step (sparse LU stage solves).

Bounds: the EREM steps replay the oracle's Leja schedules (FP64 1e-11;
FP32-bulk free-running 1e-5, on the increment too).  A CG stopped at
||r|| <= tol ||b|| is within 10 tol ||b|| / lambda_min(A) of the solution
(lambda_min of the SPD pressure matrix by shift-invert Lanczos); a stage solve
of ROS2 within ||A^-1||_2 10 tol ||rhs||, where the stage matrix
I/(tau gamma) - J is strictly diagonally dominant by rows and by columns, so
||A^-1||_2 <= sqrt(||A^-1||_1 ||A^-1||_inf) <= 1 / min(row margin, column
margin).  The oracle takes a few minutes on the host."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import cases as C
import workloads as W
from oracle import fv, timestep as ts

pytestmark = pytest.mark.gpu

N1 = 1024
STEPS = 2
CG_TOL = 1e-13
STAGE_TOL = 1e-12


@pytest.fixture(scope="module")
def run():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    wl = W.coupled2d(N1)
    g = fv.Grid(2, N1, N1)
    base = fv.Physics(head_left=wl.head_drop, head_right=0.0, T_inflow=wl.T_inflow, fluid_model=1)
    p0 = ts.pressure_solve_direct(g, base, wl.lnk, wl.T0)
    U = fv.darcy_fluxes(g, base, wl.lnk, p0, wl.T0)[0][:, :, 0].sum()
    rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), U)
    ph = fv.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 1)
    T = wl.T0.copy()
    ps, scheds, Ts = [], [], [T.copy()]
    for _ in range(STEPS):
        T, p, res = ts.sequential_step(g, ph, wl.lnk, wl.phi, wl.lam, T, None, wl.dt)
        assert res.converged
        ps.append(p)
        scheds.append(res.schedule)
        Ts.append(T.copy())
    phys = E.Physics(ph.rhoc_f, ph.rhoc_s, ph.head_left, ph.head_right, ph.T_inflow, 1)
    return E, wl, g, ph, phys, ps, scheds, Ts


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _steps(E, wl, phys, ps, precision, scheds=None):
    got_s = []
    with E.Context(2, N1, N1, physics=phys, precision=precision) as ctx:
        T = _t(wl.T0)
        for k in range(STEPS):
            opts = E.leja_opts(replay=scheds[k]) if scheds else None
            st = ctx.erem_step(T, wl.dt, _t(ps[k]), _t(wl.lnk), _t(wl.phi), _t(wl.lam), opts=opts)
            got_s.append(st.schedule)
        return T.cpu().numpy(), got_s


@pytest.mark.timeout(1800)
def test_coupled_1024_fp64_with_oracle_pressure(run):
    E, wl, g, ph, phys, ps, scheds, Ts = run
    got, got_s = _steps(E, wl, phys, ps, "fp64", scheds)
    assert got_s == scheds
    assert C.rel_l2(got, Ts[-1]) < 1e-11
    assert C.rel_l2(got - wl.T0, Ts[-1] - wl.T0) < 1e-10


@pytest.mark.timeout(1800)
def test_coupled_1024_fp32_bulk_with_oracle_pressure(run):
    E, wl, g, ph, phys, ps, scheds, Ts = run
    got, got_s = _steps(E, wl, phys, ps, "fp32_bulk")
    assert C.rel_l2(got, Ts[-1]) < 1e-5
    assert C.rel_l2(got - wl.T0, Ts[-1] - wl.T0) < 1e-5
    assert all(a[0] == b[0] and max(abs(x - y) for x, y in zip(a[1:], b[1:])) <= 2
               for a, b in zip(got_s, scheds))


@pytest.mark.timeout(1800)
def test_coupled_1024_gpu_pressure_in_the_loop(run):
    E, wl, g, ph, phys, ps, scheds, Ts = run
    bound = 0.0
    for k in range(STEPS):
        A, b = fv.pressure_system(g, ph, wl.lnk, Ts[k])
        lam_min = spla.eigsh(A.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
        assert lam_min > 0
        bound = max(bound, 10 * CG_TOL * np.linalg.norm(b) / lam_min / np.linalg.norm(ps[k]))
    with E.Context(2, N1, N1, physics=phys) as ctx:
        T = _t(wl.T0)
        p = _t(fv.linear_head_guess(g, ph))
        for k in range(STEPS):
            st = ctx.pressure_solve(_t(wl.lnk), T, p, tol=CG_TOL, maxit=20000)
            assert st.lin_resid <= CG_TOL
            if k == 0:
                assert C.rel_l2(p.cpu().numpy(), ps[0]) < 2 * bound
            ctx.erem_step(T, wl.dt, p, _t(wl.lnk), _t(wl.phi), _t(wl.lam),
                          opts=E.leja_opts(replay=scheds[k]))
        got = T.cpu().numpy()
    inc = np.linalg.norm(Ts[-1] - wl.T0) / np.linalg.norm(Ts[-1])
    assert C.rel_l2(got, Ts[-1]) < max(1e-11, 10 * STEPS * bound * inc), bound


def _inverse_norm_bound(A):
    """1 / min(row margin, column margin) of a matrix that is strictly
    diagonally dominant by rows and by columns (asserted)."""
    A = sp.csr_matrix(A)
    d = np.abs(A.diagonal())
    off_r = np.asarray(abs(A).sum(axis=1)).ravel() - d
    off_c = np.asarray(abs(A).sum(axis=0)).ravel() - d
    m = min((d - off_r).min(), (d - off_c).min())
    assert m > 0
    return 1.0 / m


@pytest.mark.timeout(1800)
def test_coupled_1024_ros2_step_matches_oracle(run):
    E, wl, g, ph, phys, ps, scheds, Ts = run
    prob = ts.heat_problem(g, ph, wl.lnk, wl.phi, wl.lam, ps[0], wl.T0)
    ref = ts.ros2_step(prob, wl.T0, wl.dt)
    A = ts.stage_matrix(prob.J(wl.T0), wl.dt, ts.ROS2_GAMMA)
    inv = _inverse_norm_bound(A)
    G = prob.G(wl.T0)
    inc = ref - wl.T0
    # each of the two stages: error <= 10 tol ||rhs|| ||A^-1||, rhs ~ G;
    # combined with the weights b_i and 1/gamma (a factor 3, as on small grids)
    bound = 10 * STAGE_TOL * np.linalg.norm(G) * inv * 3.0 / np.linalg.norm(inc)
    with E.Context(2, N1, N1, physics=phys) as ctx:
        T = _t(wl.T0)
        st = ctx.rosm_step(T, wl.dt, E.EREM_ROS2, _t(ps[0]), _t(wl.lnk), _t(wl.phi), _t(wl.lam),
                           lin_tol=STAGE_TOL, maxit=20000)
        got = T.cpu().numpy()
    assert st.lin_resid <= STAGE_TOL
    err = np.linalg.norm((got - wl.T0) - inc) / np.linalg.norm(inc)
    assert err <= max(bound, 1e-11), (err, bound)

"""Pins of the oracle's non-autonomous EREM (oracle/nonauto.py, eq. ``nEERMg``):
phi_2 divided differences against 120-digit arithmetic, D_t G against
central differences of G in the inflow temperature, exactness of one step
for a forcing linear in t against the dense exponential of the augmented
system (y, t, 1), the scalar closed form, reduction to the autonomous step,
and the observed order for a sinusoidal inflow temperature."""
import math
from dataclasses import replace

import numpy as np
import pytest
import scipy.linalg as sla

import cases as C
from oracle import fv, leja, nonauto as NA, timestep as ts
from oracle.leja import LejaOptions


def _mp_phi2_dd(xi, c, gamma):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 120

    def phi2(z):
        return (mp.exp(z) - 1 - z) / z**2 if z != 0 else mp.mpf(1) / 2

    xs = [mp.mpf(float(x)) for x in xi]
    col = [phi2(mp.mpf(c) + mp.mpf(gamma) * x) for x in xs]
    out = [col[0]]
    for j in range(1, len(xs)):
        col = [(col[i + 1] - col[i]) / (xs[i + j] - xs[i]) for i in range(len(col) - 1)]
        out.append(col[0])
    return np.array([float(v) for v in out])


@pytest.mark.parametrize("c,gamma", [(-3.0, 1.5), (-20.0, 10.0), (-0.5, 0.25), (-7.0, 2.0)])
def test_phi2_divided_differences_vs_high_precision(c, gamma):
    xi = leja.leja_points(40)
    got = NA.phi2_divided_differences(xi, c, gamma)
    want = _mp_phi2_dd(xi, c, gamma)
    big = np.abs(want) > 1e-250
    assert np.max(np.abs(got[big] - want[big]) / np.abs(want[big])) < 1e-10
    # d_0 = phi_2(beta) in closed form
    z = c + 2.0 * gamma
    assert got[0] == pytest.approx((math.expm1(z) - z) / z**2 if z != 0 else 0.5, rel=1e-13)


@pytest.mark.parametrize("fm", [0, 1])
def test_inflow_sensitivity_is_the_derivative_of_G(fm):
    case = C.random_case(2, 9, 7, seed=3, fluid_model=fm)
    pb = case.problem(case.T0)
    T_in, h = 70.0, 1e-3
    Gp = replace(pb, phys=replace(pb.phys, T_inflow=T_in + h)).G(case.T0)
    Gm = replace(pb, phys=replace(pb.phys, T_inflow=T_in - h)).G(case.T0)
    ph = replace(pb.phys, T_inflow=T_in)
    got = NA.inflow_sensitivity(pb.grid, ph, pb.phi, pb.lam, pb.fluxes, T_in)
    fd = (Gp - Gm) / (2 * h)
    assert np.max(np.abs(got - fd)) < 1e-7 * np.max(np.abs(fd))
    first, _ = fv.boundary_cells_x(pb.grid)
    mask = np.ones(pb.grid.n, bool)
    mask[first] = False
    assert np.all(got[mask] == 0.0) and np.all(got[first] > 0.0)


def _augmented_exact(J, v, w, y0, tau):
    # y' = J y + v + t w, t' = 1 as one linear system in (y, t, 1)
    n = y0.size
    A = np.zeros((n + 2, n + 2))
    A[:n, :n] = J
    A[:n, n] = w
    A[:n, n + 1] = v
    A[n, n + 1] = 1.0
    z0 = np.concatenate([y0, [0.0, 1.0]])
    return (sla.expm(tau * A) @ z0)[:n]


@pytest.mark.parametrize("tau", [0.02, 0.3])
def test_step_is_exact_for_a_forcing_linear_in_time(tau):
    # G(T, t) = J T + b(t) with b linear in t: the non-autonomous EREM step
    # is the exact flow; at 1e-13 the Leja truncation is far below it
    case = C.heat2d_rect(7, 6)
    pb = case.problem(case.T0)
    T0 = case.T0 + np.random.default_rng(2).uniform(0, 30, case.n)
    J = pb.J(T0).toarray()
    rate = 150.0
    T1, res = NA.erem_step_forced(pb, T0, tau, 60.0, rate, LejaOptions(tol_a=1e-13, tol_r=1e-13))
    ph = replace(pb.phys, T_inflow=60.0)
    pb60 = replace(pb, phys=ph)
    w = rate * NA.inflow_sensitivity(pb.grid, ph, pb.phi, pb.lam, pb.fluxes, 60.0)
    v = pb60.G(T0) - J @ T0   # b(t_n)
    want = _augmented_exact(J, v, w, T0, tau)
    assert res.converged
    assert np.linalg.norm(T1 - want) < 1e-10 * np.linalg.norm(want - T0)
    # and across substeps: two and four pieces give the same flow
    for s in (2, 4):
        sched = [s] + [res.degrees[0] + 10] * s + [res.degree_phi2 + 10]
        Ts, _ = NA.erem_step_forced(pb, T0, tau, 60.0, rate, LejaOptions(replay=sched))
        assert np.linalg.norm(Ts - want) < 1e-10 * np.linalg.norm(want - T0)


def test_scalar_closed_form():
    # y' = lam y + a + b t on one cell: y(tau) = e^{lam tau} y0 + tau phi_1 (lam y0 + a) + tau^2 phi_2 b
    lam_, a, b, y0, tau = -3.0, 2.0, 5.0, 1.5, 0.4
    J = np.array([[lam_]])
    res = NA.phi12_leja(J, np.array([lam_ * y0 + a]), np.array([b]), tau, abs(y0),
                        LejaOptions(tol_a=1e-14, tol_r=1e-14))
    z = lam_ * tau
    phi1 = math.expm1(z) / z
    phi2 = (math.expm1(z) - z) / z**2
    exact = tau * phi1 * (lam_ * y0 + a) + tau**2 * phi2 * b
    assert res.value[0] == pytest.approx(exact, rel=1e-12)
    # the solution of the ODE itself
    yt = math.exp(z) * y0 + (a / lam_ + b / lam_**2) * math.expm1(z) - b * tau / lam_
    assert y0 + res.value[0] == pytest.approx(yt, rel=1e-12)


def test_zero_rate_is_the_autonomous_step():
    case = C.heat2d(32)
    pb = case.problem(case.T0)
    T1, res = NA.erem_step_forced(pb, case.T0, case.dt, pb.phys.T_inflow, 0.0)
    T2, res2 = ts.erem_step(pb, case.T0, case.dt)
    assert res.schedule[:-1] == res2.schedule
    assert np.linalg.norm(T1 - T2) <= 1e-13 * np.linalg.norm(T2)


def test_second_order_for_a_sinusoidal_inflow():
    # T_in(t) = 60 + 20 sin(8 t) over [0, 0.4]; errors against a run with
    # 16x smaller steps fall by about 4 per halving (order 2)
    case = C.heat2d_rect(12, 10)
    pb = case.problem(case.T0)
    tin = lambda t: 60.0 + 20.0 * math.sin(8.0 * t)
    rate = lambda t: 160.0 * math.cos(8.0 * t)
    opts = LejaOptions(tol_a=1e-12, tol_r=1e-12)

    def run(nsteps):
        T = case.T0.copy()
        tau = 0.4 / nsteps
        for k in range(nsteps):
            T, _ = NA.erem_step_forced(pb, T, tau, tin(k * tau), rate(k * tau), opts)
        return T

    ref = run(64)
    errs = [np.linalg.norm(run(n) - ref) for n in (4, 8)]
    order = math.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.3, (errs, order)

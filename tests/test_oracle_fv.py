"""Pins of the oracle's finite-volume discretization (§2, §3.1): closed-form
pressure solutions, discrete mass and energy conservation, and the Jacobian
against finite differences of the right-hand side."""
import numpy as np
import pytest

import workloads as W
from oracle import fv, timestep as ts


def test_pressure_constant_k_is_linear_head():
    g = fv.Grid(2, 12, 7)
    ph = fv.Physics(head_left=3.0, head_right=1.0)
    lnk = np.full(g.n, np.log(2.5))
    p = ts.pressure_solve_direct(g, ph, lnk)
    x = g.cell_centres_x()
    np.testing.assert_allclose(p, 3.0 - 2.0 * x, rtol=0, atol=1e-13)
    vx, vy, _ = fv.darcy_fluxes(g, ph, lnk, p)
    # Darcy: v = K * (head drop) / L per unit area; face area hy = 1/7
    np.testing.assert_allclose(vx, 2.5 * 2.0 / 7, rtol=1e-13)
    assert np.abs(vy).max() < 1e-13


def test_pressure_layers_in_series_harmonic_closed_form():
    # K varies along x only: every row is a chain of resistances h/K_i, so the
    # flux per unit area is the head drop over sum_i h / K_i.
    nx, ny = 16, 3
    g = fv.Grid(2, nx, ny)
    ph = fv.Physics(head_left=1.0, head_right=0.0)
    K = np.exp(np.random.default_rng(0).normal(0, 1.5, nx))
    lnk = np.tile(np.log(K), ny)
    p = ts.pressure_solve_direct(g, ph, lnk)
    vx, vy, _ = fv.darcy_fluxes(g, ph, lnk, p)
    h = 1.0 / nx
    q = 1.0 / np.sum(h / K)
    np.testing.assert_allclose(vx, q / ny, rtol=1e-12)
    assert np.abs(vy).max() < 1e-12 * q


def test_pressure_cg_matches_direct():
    wl = W.heat2d(24)
    g = fv.Grid(2, 24, 24)
    ph = fv.Physics()
    pd = ts.pressure_solve_direct(g, ph, wl.lnk)
    pc, it, res = ts.pressure_solve_cg(g, ph, wl.lnk, tol=1e-14)
    assert res <= 1e-14 and it > 0
    np.testing.assert_allclose(pc, pd, rtol=0, atol=1e-10)


@pytest.mark.parametrize("fluid_model", [0, 1])
def test_discrete_mass_conservation(fluid_model):
    wl = W.heat2d(32, sigma=1.5)
    g = fv.Grid(2, 32, 32)
    ph = fv.Physics(fluid_model=fluid_model)
    T = np.linspace(20, 80, g.n)
    p = ts.pressure_solve_direct(g, ph, wl.lnk, T)
    if fluid_model == 0:
        vx, vy, vz = fv.darcy_fluxes(g, ph, wl.lnk, p, T)
        div = fv.cell_net_outflow(g, vx, vy, vz)
        assert np.abs(div).max() < 1e-12 * np.abs(vx).max()
    # the mass flux K rho/mu grad p balances in every cell
    A, b = fv.pressure_system(g, ph, wl.lnk, T)
    assert np.abs(A @ p - b).max() < 1e-12 * np.abs(b).max()


def _problem(dim, n, fluid_model, seed=1):
    rng = np.random.default_rng(seed)
    g = fv.Grid(dim, n, n + 1, n - 1 if dim == 3 else 1)
    ph = fv.Physics(rhoc_f=30.0, rhoc_s=25.0, T_inflow=80.0, fluid_model=fluid_model,
                    head_left=1.0, head_right=-0.5)
    lnk = rng.normal(0, 1, g.n)
    lam = rng.uniform(0.5, 3.0, g.n)
    phi = rng.uniform(0.1, 0.3, g.n)
    T = rng.uniform(20, 80, g.n)
    p = ts.pressure_solve_direct(g, ph, lnk, T)
    return g, ph, ts.heat_problem(g, ph, lnk, phi, lam, p, T), T, lam


@pytest.mark.parametrize("dim,fluid_model", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_jacobian_matches_central_differences(dim, fluid_model):
    g, ph, prob, T, _ = _problem(dim, 5, fluid_model)
    J = prob.J(T)
    rng = np.random.default_rng(7)
    for _ in range(4):
        d = rng.normal(0, 1, g.n)
        eps = 1e-4
        fd = (prob.G(T + eps * d) - prob.G(T - eps * d)) / (2 * eps)
        np.testing.assert_allclose(J @ d, fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_model_is_affine_in_T(dim):
    # fluid_model 0: G(T) = J T + G(0) exactly, so J holds every T-dependence
    g, ph, prob, T, _ = _problem(dim, 6, 0)
    J = prob.J(T)
    np.testing.assert_allclose(prob.G(T), J @ T + prob.G(np.zeros(g.n)), rtol=1e-12,
                               atol=1e-12 * np.abs(prob.G(T)).max())


@pytest.mark.parametrize("dim,fluid_model", [(2, 0), (3, 1)])
def test_discrete_energy_conservation(dim, fluid_model):
    # interior face fluxes cancel: sum_i C_i |Omega_i| G_i equals the heat that
    # enters through the x = 0 face minus what leaves through x = 1
    g, ph, prob, T, lam = _problem(dim, 6, fluid_model)
    total = np.sum(fv.capacity(g, ph, prob.phi) * prob.G(T))
    vx = prob.fluxes[0]
    first, last = fv.boundary_cells_x(g)
    X = fv.advected(T, ph)
    F0 = ph.rhoc_f * vx[:, :, 0].reshape(-1)
    F1 = ph.rhoc_f * vx[:, :, -1].reshape(-1)
    X_in = fv.advected(np.array(ph.T_inflow), ph)
    cond0 = lam[first] * g.face_area[0] / (g.h[0] / 2) * (ph.T_inflow - T[first])
    boundary = np.sum(cond0 + F0 * np.where(F0 > 0, X_in, X[first])) - np.sum(F1 * X[last])
    assert total == pytest.approx(boundary, rel=1e-12, abs=1e-12 * np.abs(cond0).sum())


def test_pure_conduction_rows_sum_to_zero_away_from_dirichlet():
    g = fv.Grid(3, 5, 4, 3)
    ph = fv.Physics(head_left=0.0, head_right=0.0)
    rng = np.random.default_rng(2)
    lnk = rng.normal(size=g.n)
    p = np.zeros(g.n)
    prob = ts.heat_problem(g, ph, lnk, np.full(g.n, 0.2), rng.uniform(1, 2, g.n), p)
    J = prob.J(np.full(g.n, 30.0))
    rows = np.asarray(J.sum(axis=1)).reshape(-1)
    first, _ = fv.boundary_cells_x(g)
    mask = np.ones(g.n, bool)
    mask[first] = False
    assert np.abs(rows[mask]).max() < 1e-12 * np.abs(J.diagonal()).max()
    assert np.all(rows[first] < 0)
    # off-diagonal entries of the conduction operator are symmetric after
    # scaling by the capacity
    C = fv.capacity(g, ph, prob.phi)
    S = (J.multiply(C[:, None])).toarray()
    np.testing.assert_allclose(S, S.T, atol=1e-12 * np.abs(S).max())

"""Pins of the oracle's adjoint (oracle/adjoint.py): the frozen-schedule
forward equals the oracle's EREM step, the step adjoint is the transpose of
the step built column by column, and the gradients with respect to T^0 and
ln K agree with central finite differences of the frozen forward (the
schedules and spectral intervals held at their forward values, the pressure
re-solved for every perturbed ln K)."""
import numpy as np
import pytest
import scipy.sparse as sp

import cases as C
from oracle import adjoint as A, fv, leja, timestep as ts


def _setup(shape, steps=3, seed=0):
    case = C.heat2d_rect(*shape) if len(shape) == 2 else C.random_case(3, *shape, seed=seed)
    g, ph = case.grid, case.phys
    rng = np.random.default_rng(seed + 5)
    obs = np.sort(rng.choice(g.n, size=min(6, g.n), replace=False))
    data = case.T0[obs] + 5.0 * rng.standard_normal(obs.size)
    return case, g, ph, obs, data, steps


def _frozen_L(case, g, ph, lnk, T0, frozen, obs, data):
    base = fv.Physics(head_left=ph.head_left, head_right=ph.head_right, fluid_model=0)
    p = ts.pressure_solve_direct(g, base, lnk, None)
    tr = A.forward(lambda: ts.heat_problem(g, ph, lnk, case.phi, case.lam, p), T0, case.dt,
                   len(frozen), frozen=frozen)
    return A.misfit(tr.T[-1], obs, data)


def test_frozen_forward_matches_the_oracle_step():
    case, g, ph, obs, data, steps = _setup((12, 10))
    tr = A.forward(lambda: case.problem(), case.T0, case.dt, steps)
    T = case.T0.copy()
    for n in range(steps):
        T, res = ts.erem_step(case.problem(), T, case.dt)
        assert res.schedule == tr.steps[n].schedule
        assert np.linalg.norm(tr.T[n + 1] - T) < 1e-12 * np.linalg.norm(T)


def test_step_adjoint_is_the_transpose_of_the_step():
    case, g, ph, obs, data, _ = _setup((4, 3))
    pb = case.problem()
    J = sp.csr_matrix(pb.J(case.T0))
    b = pb.G(np.zeros(g.n))
    alpha, beta = leja.gershgorin_interval(J, case.dt)
    fr = A.FrozenStep([2, 9, 7], alpha, beta)
    xi = leja.cached_leja_points(150)
    zero = A.step_forward(J, b, np.zeros(g.n), case.dt, fr, xi)
    M = np.column_stack([A.step_forward(J, b, e, case.dt, fr, xi) - zero for e in np.eye(g.n)])
    lam = np.random.default_rng(1).standard_normal(g.n)
    got = A.step_adjoint(J, b, case.T0, case.dt, fr, lam, xi)
    assert np.max(np.abs(got - M.T @ lam)) < 1e-12 * np.max(np.abs(M.T @ lam))


@pytest.mark.parametrize("shape", [(10, 8), (5, 4, 4)])
def test_t0_gradient_matches_central_differences(shape):
    case, g, ph, obs, data, steps = _setup(shape)
    L, gT0, _, tr = A.gradients(g, ph, case.lnk, case.phi, case.lam, case.T0, case.dt, steps,
                                obs, data, p=case.p)
    rng = np.random.default_rng(2)
    for _ in range(4):
        dirn = rng.standard_normal(g.n)
        h = 1e-4
        Lp = _frozen_L(case, g, ph, case.lnk, case.T0 + h * dirn, tr.steps, obs, data)
        Lm = _frozen_L(case, g, ph, case.lnk, case.T0 - h * dirn, tr.steps, obs, data)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gT0 @ dirn) < 1e-7 * max(abs(fd), 1e-3 * L)


@pytest.mark.parametrize("shape", [(10, 8), (5, 4, 4)])
def test_lnk_gradient_matches_central_differences(shape):
    case, g, ph, obs, data, steps = _setup(shape)
    base = fv.Physics(head_left=ph.head_left, head_right=ph.head_right, fluid_model=0)
    p = ts.pressure_solve_direct(g, base, case.lnk, None)
    L, _, glnk, tr = A.gradients(g, ph, case.lnk, case.phi, case.lam, case.T0, case.dt, steps,
                                 obs, data, p=p)
    rng = np.random.default_rng(3)
    for _ in range(4):
        dirn = rng.standard_normal(g.n)
        h = 1e-5
        Lp = _frozen_L(case, g, ph, case.lnk + h * dirn, case.T0, tr.steps, obs, data)
        Lm = _frozen_L(case, g, ph, case.lnk - h * dirn, case.T0, tr.steps, obs, data)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - glnk @ dirn) < 1e-5 * max(abs(fd), 1e-3 * L), (fd, glnk @ dirn)


def test_lnk_gradient_of_a_flux_functional():
    # the pressure-adjoint part alone: L = sum_sigma c_sigma F_sigma
    case, g, ph, obs, data, _ = _setup((9, 7))
    base = fv.Physics(head_left=ph.head_left, head_right=ph.head_right, fluid_model=0)
    rng = np.random.default_rng(4)
    fg = A._face_grad_zero(g)
    for ax in fg.interior:
        fg.interior[ax] = rng.standard_normal(fg.interior[ax].size)
    fg.f0 = rng.standard_normal(fg.f0.size)
    fg.f1 = rng.standard_normal(fg.f1.size)

    def L_of(lnk):
        p = ts.pressure_solve_direct(g, base, lnk, None)
        vx, vy, _ = fv.darcy_fluxes(g, ph, lnk, p)
        F = {ax: ph.rhoc_f * v for ax, _, _, v in fv._face_families(g, vx, vy, None)}
        return (sum(float(fg.interior[ax] @ F[ax]) for ax in F)
                + float(fg.f0 @ (ph.rhoc_f * vx[:, :, 0].reshape(-1)))
                + float(fg.f1 @ (ph.rhoc_f * vx[:, :, -1].reshape(-1))))

    p = ts.pressure_solve_direct(g, base, case.lnk, None)
    grad = A.lnk_gradient(g, ph, case.lnk, p, fg)
    for _ in range(3):
        dirn = rng.standard_normal(g.n)
        h = 1e-5
        fd = (L_of(case.lnk + h * dirn) - L_of(case.lnk - h * dirn)) / (2 * h)
        assert abs(fd - grad @ dirn) < 1e-6 * max(abs(fd), 1.0)


def test_lnk_gradient_through_substeps():
    # frozen two- and three-substep schedules: the J w_k uses of later substeps
    case, g, ph, obs, data, _ = _setup((8, 7))
    pb = case.problem()
    J = sp.csr_matrix(pb.J(case.T0))
    alpha, beta = leja.gershgorin_interval(J, case.dt)
    frozen = [A.FrozenStep([2, 30, 25], alpha, beta), A.FrozenStep([3, 20, 18, 15], alpha, beta)]
    base = fv.Physics(head_left=ph.head_left, head_right=ph.head_right, fluid_model=0)
    p = ts.pressure_solve_direct(g, base, case.lnk, None)
    L, gT0, glnk, _ = A.gradients(g, ph, case.lnk, case.phi, case.lam, case.T0, case.dt, 2, obs,
                                  data, frozen=frozen, p=p)
    rng = np.random.default_rng(6)
    for _ in range(3):
        dirn = rng.standard_normal(g.n)
        h = 1e-5
        fd = (_frozen_L(case, g, ph, case.lnk + h * dirn, case.T0, frozen, obs, data)
              - _frozen_L(case, g, ph, case.lnk - h * dirn, case.T0, frozen, obs, data)) / (2 * h)
        assert abs(fd - glnk @ dirn) < 1e-5 * max(abs(fd), 1e-3 * L), (fd, glnk @ dirn)
        fdT = (_frozen_L(case, g, ph, case.lnk, case.T0 + 1e-4 * dirn, frozen, obs, data)
               - _frozen_L(case, g, ph, case.lnk, case.T0 - 1e-4 * dirn, frozen, obs, data)) / 2e-4
        assert abs(fdT - gT0 @ dirn) < 1e-7 * max(abs(fdT), 1e-3 * L)

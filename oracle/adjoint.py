"""Adjoint of EREM steps with real Leja phi_1 (oracle): gradients of a
temperature misfit with respect to T^0 and to ln K.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The forward map is the one of ``oracle.timestep.erem_step`` (eq. ``EERM``
with the Newton form of eq. ``newt``, §4.2) for the linear fluid model, where
G(T) = J T + b exactly and the Darcy field comes from one steady pressure
solve.  The Leja schedule (substep count, degrees) and the spectral interval
[alpha, beta] of every step are frozen at their forward values: the stopping
test is a discrete decision and the interval a Gershgorin bound, neither is
differentiated.  With them frozen a step is

    w_0 = 0,  u_k = G + J w_k,  w_{k+1} = w_k + P_k u_k,  T^{n+1} = T^n + w_S,

P_k = delta sum_m d_m prod_{i<m} B_i, B_i = (delta J - c I)/gamma - xi_i I
(c, gamma the focal values of the substep).  Its transpose is the same
polynomial in J^T; evaluated by the Horner recurrence
s_M = d_M mu, s_j = d_j mu + B_j^T s_{j+1}, it gives P_k^T mu = delta s_0,
and the pairs (s_{j+1}, q_j) with the forward Newton vectors q_j give the
derivative of P_k u_k with respect to J (factor delta^2 / gamma).

Every use of J on a vector x with adjoint vector y contributes to the
derivative with respect to the upwind face fluxes F = (rho c)_f v (§3.1):
(y_R / C_R - y_L / C_L) x_up on an interior face, y x / C on the x = 0 face
when it is an outflow, -y x / C on the x = 1 face; the constant part b of G
contributes y X(T_inflow) / C on an inflowing x = 0 face.  The fluxes depend
on ln K through the harmonic transmissibilities and the pressure; one
adjoint pressure solve (the TPFA matrix is symmetric) carries the gradient
through p.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fv, leja
from .timestep import heat_problem, pressure_solve_direct


@dataclass
class FrozenStep:
    schedule: list          # [S, m_1, .., m_S]
    alpha: float
    beta: float


@dataclass
class Trajectory:
    T: list = field(default_factory=list)        # T^0 .. T^N
    steps: list = field(default_factory=list)    # FrozenStep per step


def _substep_data(fr: FrozenStep, tau: float, xi_all):
    S = fr.schedule[0]
    c, gamma = leja.focal_map(fr.alpha, fr.beta)
    M = max(fr.schedule[1:])
    xi = xi_all[: M + 1]
    d = leja.phi1_divided_differences(xi, c / S, gamma / S)
    return S, tau / S, c / S, gamma / S, xi, d


def step_forward(J, b, T, tau, fr: FrozenStep, xi_all, record=False):
    """One EREM step with frozen schedule and interval (the Newton form of
    eq. ``newt``).  With record, also returns for each substep the w_k before
    it and its Newton vectors q_0..q_m."""
    S, delta, cs, gs, xi, d = _substep_data(fr, tau, xi_all)
    G = J @ T + b
    w = np.zeros_like(T)
    rec = []
    for k in range(S):
        u = G if k == 0 else G + J @ w
        q = [u]
        for m in range(1, fr.schedule[1 + k] + 1):
            q.append((delta * (J @ q[-1]) - cs * q[-1]) / gs - xi[m - 1] * q[-1])
        if record:
            rec.append((w.copy(), q))
        w = w + delta * sum(d[m] * q[m] for m in range(len(q)))
    return (T + w, (G, rec)) if record else T + w


def forward(problem_of, T0, tau, n_steps, opts=None, frozen=None):
    """n_steps EREM steps; the schedules and intervals are taken free (the
    stopping test of §4.2) or from ``frozen``.  problem_of() gives the
    HeatProblem (J, b fixed: linear fluid model)."""
    pb = problem_of()
    J = sp.csr_matrix(pb.J(T0))
    b = pb.G(np.zeros_like(T0))
    xi_all = leja.cached_leja_points(leja.LejaOptions().m_max if opts is None else opts.m_max)
    tr = Trajectory(T=[np.asarray(T0, np.float64).copy()])
    T = tr.T[0]
    for n in range(n_steps):
        if frozen is None:
            alpha, beta = leja.gershgorin_interval(J, tau)
            res = leja.phi1_leja(J, J @ T + b, tau, float(np.max(np.abs(T))), opts)
            fr = FrozenStep(res.schedule, alpha, beta)
        else:
            fr = frozen[n]
        xi_all = leja.cached_leja_points(max(max(fr.schedule[1:]), 150))
        T = step_forward(J, b, T, tau, fr, xi_all)
        tr.T.append(T)
        tr.steps.append(fr)
    return tr


def misfit(T, obs, data):
    r = T[obs] - data
    return float(r @ r)


# --------------------------------------------------------------------------
# derivative with respect to the face fluxes of one use of J (or of b)
# --------------------------------------------------------------------------
@dataclass
class FaceGrad:
    """dL/dF on the faces: interior families (axis, left, right, value) and
    the x = 0 / x = 1 boundary faces (per boundary cell)."""
    interior: dict
    f0: np.ndarray
    f1: np.ndarray


def _face_grad_zero(g):
    interior = {ax: np.zeros(L.size) for ax, L, R in fv.interior_faces(g)}
    first, last = fv.boundary_cells_x(g)
    return FaceGrad(interior, np.zeros(first.size), np.zeros(last.size))


def accumulate_j_use(g, phys, cap, fluxes, y, x, fgrad: FaceGrad, scale=1.0):
    """fgrad += scale * d(y^T J x)/dF for every face flux F (linear model)."""
    vx, vy, vz = fluxes
    yc = y / cap
    for ax, L, R, v in fv._face_families(g, vx, vy, vz):
        F = phys.rhoc_f * v
        x_up = np.where(F >= 0, x[L], x[R])
        fgrad.interior[ax] += scale * (yc[R] - yc[L]) * x_up
    first, last = fv.boundary_cells_x(g)
    F0 = phys.rhoc_f * vx[:, :, 0].reshape(-1)
    fgrad.f0 += scale * np.where(F0 > 0, 0.0, yc[first] * x[first])
    fgrad.f1 += scale * (-yc[last] * x[last])


def accumulate_b_use(g, phys, cap, fluxes, y, fgrad: FaceGrad):
    """fgrad += d(y^T b)/dF (the inflow of X(T_inflow) through x = 0)."""
    vx = fluxes[0]
    first, _ = fv.boundary_cells_x(g)
    F0 = phys.rhoc_f * vx[:, :, 0].reshape(-1)
    X_in = fv.advected(np.full(first.shape, phys.T_inflow), phys)
    fgrad.f0 += np.where(F0 > 0, (y / cap)[first] * X_in, 0.0)


# --------------------------------------------------------------------------
# backward through the steps
# --------------------------------------------------------------------------
def step_adjoint(J, b, T, tau, fr: FrozenStep, lam, xi_all, face=None):
    """dL/dT^n from dL/dT^{n+1} = lam for one frozen step; with ``face`` =
    (g, phys, cap, fluxes, fgrad) the face-flux derivative is accumulated."""
    S, delta, cs, gs, xi, d = _substep_data(fr, tau, xi_all)
    _, (G, rec) = step_forward(J, b, T, tau, fr, xi_all, record=True)
    JT = J.T.tocsr()
    mu = lam.copy()
    G_adj = np.zeros_like(T)
    for k in range(S - 1, -1, -1):
        w_k, q = rec[k]
        mk = len(q) - 1
        s = d[mk] * mu
        for j in range(mk - 1, -1, -1):
            if face is not None:
                accumulate_j_use(*face[:4], s, q[j], face[4], scale=delta * delta / gs)
            s = d[j] * mu + (delta * (JT @ s) - cs * s) / gs - xi[j] * s
        z = delta * s
        G_adj += z
        if face is not None and k > 0:
            accumulate_j_use(*face[:4], z, w_k, face[4])
        mu = mu + JT @ z
    if face is not None:
        accumulate_j_use(*face[:4], G_adj, T, face[4])
        accumulate_b_use(*face[:3], face[3], G_adj, face[4])
    return lam + JT @ G_adj


def gradients(g, phys, lnk, phi, lam_field, T0, tau, n_steps, obs, data, opts=None, frozen=None,
              p=None):
    """Misfit L = sum_o (T^N_o - data_o)^2 after n_steps and its gradients
    (dL/dT^0, dL/dlnK), with the schedules and intervals frozen (free on the
    forward run unless ``frozen`` is given).  The pressure is the steady TPFA
    solution for lnK (direct solve) unless ``p`` is given."""
    lnk = np.asarray(lnk, np.float64).reshape(-1)
    if p is None:
        base = fv.Physics(head_left=phys.head_left, head_right=phys.head_right,
                          T_inflow=phys.T_inflow, fluid_model=0)
        p = pressure_solve_direct(g, base, lnk, None)
    fluxes = fv.darcy_fluxes(g, phys, lnk, p)

    def problem_of():
        return heat_problem(g, phys, lnk, phi, lam_field, p)

    tr = forward(problem_of, T0, tau, n_steps, opts, frozen)
    pb = problem_of()
    J = sp.csr_matrix(pb.J(T0))
    b = pb.G(np.zeros_like(T0))
    cap = fv.capacity(g, phys, phi)
    fgrad = _face_grad_zero(g)
    lam = np.zeros_like(T0)
    lam[obs] = 2.0 * (tr.T[-1][obs] - data)
    L = misfit(tr.T[-1], obs, data)
    for n in range(n_steps - 1, -1, -1):
        fr = tr.steps[n]
        xi_all = leja.cached_leja_points(max(max(fr.schedule[1:]), 150))
        lam = step_adjoint(J, b, tr.T[n], tau, fr, lam, xi_all, (g, phys, cap, fluxes, fgrad))
    return L, lam, lnk_gradient(g, phys, lnk, p, fgrad), tr


def lnk_gradient(g, phys, lnk, p, fgrad: FaceGrad):
    """dL/dlnK from dL/dF through the Darcy fluxes F = (rho c)_f v(lnK, p)
    and the steady pressure A(lnK) p = q(lnK) (one adjoint solve)."""
    k = np.exp(lnk)
    h = g.h
    area = g.face_area
    rc = phys.rhoc_f
    first, last = fv.boundary_cells_x(g)
    # dL/dp, then A mu = dL/dp (A symmetric)
    dLdp = np.zeros(g.n)
    ups_int = {}
    for ax, L, R in fv.interior_faces(g):
        ups = fv.tpfa_interior(k[L], k[R], area[ax], h[ax] / 2, h[ax] / 2)
        ups_int[ax] = (L, R, ups)
        gv = rc * fgrad.interior[ax]
        np.add.at(dLdp, L, gv * ups)
        np.add.at(dLdp, R, -gv * ups)
    ups0 = fv.tpfa_dirichlet(k[first], area[0], h[0] / 2)
    ups1 = fv.tpfa_dirichlet(k[last], area[0], h[0] / 2)
    np.add.at(dLdp, first, -rc * fgrad.f0 * ups0)
    np.add.at(dLdp, last, rc * fgrad.f1 * ups1)
    base = fv.Physics(head_left=phys.head_left, head_right=phys.head_right, fluid_model=0)
    A, _ = fv.pressure_system(g, base, lnk, None)
    mu = spla.spsolve(A.tocsc(), dLdp)
    # dL/dlnK_c = sum over the faces of c of Phi_sigma d ups_sigma / dlnK_c
    out = np.zeros(g.n)
    for ax, (L, R, ups) in ups_int.items():
        dp = p[L] - p[R]
        phi_s = dp * (rc * fgrad.interior[ax] - (mu[L] - mu[R]))
        den = k[L] + k[R]
        np.add.at(out, L, phi_s * ups * k[R] / den)
        np.add.at(out, R, phi_s * ups * k[L] / den)
    np.add.at(out, first, ups0 * (phys.head_left - p[first]) * (rc * fgrad.f0 + mu[first]))
    np.add.at(out, last, ups1 * (p[last] - phys.head_right) * (rc * fgrad.f1 - mu[last]))
    return out

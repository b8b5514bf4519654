"""Non-autonomous EREM (eq. ``nEERMg`` of §3.2) with phi_1 and phi_2 by real
Leja interpolation (§4.2) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For y' = f(y, t), after the transformation to an autonomous system (§3.2),
one step is

    y^{n+1} = y^n + tau phi_1(tau J) f(y^n, t_n) + tau^2 phi_2(tau J) D_t f(y^n, t_n),

J = D_y f(y^n, t_n), phi_2(z) = (e^z - 1 - z) / z^2.  Here the time
dependence is that of the inflow temperature T_in(t) of the heat problem:
D_t G = T_in'(t) dG/dT_in, nonzero on the x = 0 cells only.

Leja form.  Both products are Newton interpolations on the Leja points of
the interval of tau J (§4.2): the divided differences of phi_2 are the first
column of phi_2(L), L = c I + gamma L_hat, as for phi_1, read off the
exponential of [[L, e_1, 0], [0, 0, 1], [0, 0, 0]].  Substeps (when m_max
terms do not meet the stopping test): the linear ODE y' = J y + v + t w on
[0, tau] is advanced over s pieces of length delta = tau / s; piece k starts
at t = k delta from y_k and adds delta phi_1(delta J)(J y_k + v + k delta w)
+ delta^2 phi_2(delta J) w, the last term the same for every piece.  The
phi_2 interpolation takes the same stopping rule on its increment
delta^2 d_j q_j; failing either doubles s.  Schedules are
[s, m_1..m_s, m_phi2].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import fv
from .leja import (LejaOptions, cached_leja_points, expm_taylor, focal_map, gershgorin_interval,
                   phi1_divided_differences, weighted_norm)


def phi2_divided_differences(xi, c: float, gamma: float) -> np.ndarray:
    """d_j = phi_2[xi_0, ..., xi_j] of xi -> phi_2(c + gamma xi): the first
    column of phi_2(L), L = c I + gamma L_hat, which is the upper-right
    column of exp([[L, e_1, 0], [0, 0, 1], [0, 0, 0]]) (the exponential of
    that block matrix carries sum_k L^k / (k+2)! there)."""
    xi = np.asarray(xi, np.float64)
    m1 = xi.size
    L = c * np.eye(m1) + gamma * (np.diag(xi) + np.diag(np.ones(m1 - 1), -1))
    A = np.zeros((m1 + 2, m1 + 2))
    A[:m1, :m1] = L
    A[0, m1] = 1.0
    A[m1, m1 + 1] = 1.0
    return expm_taylor(A)[:m1, m1 + 1].copy()


def inflow_sensitivity(g: fv.Grid, phys: fv.Physics, phi, lam, fluxes, T_in: float):
    """dG/dT_in: the x = 0 faces carry the Dirichlet conduction
    condD (T_in - T) and, where they flow in, F0 X(T_in) (§3.1), both
    divided by the cell's capacity."""
    vx, _, _ = fluxes
    lam = np.asarray(lam, np.float64).reshape(-1)
    first, _ = fv.boundary_cells_x(g)
    condD = fv.tpfa_dirichlet(lam[first], g.face_area[0], g.h[0] / 2)
    F0 = phys.rhoc_f * vx[:, :, 0].reshape(-1)
    dX = fv.advected_dT(np.full(first.shape, T_in), phys)
    out = np.zeros(g.n)
    np.add.at(out, first, condD + np.where(F0 > 0, F0 * dX, 0.0))
    return out / fv.capacity(g, phys, phi)


@dataclass
class Phi12Result:
    value: np.ndarray          # tau phi_1(tau J) v + tau^2 phi_2(tau J) w
    substeps: int
    degrees: list = field(default_factory=list)   # phi_1 degree of each piece
    degree_phi2: int = 0
    converged: bool = True

    @property
    def schedule(self):
        return [self.substeps] + list(self.degrees) + [self.degree_phi2]


def _newton(J, u, delta, c, gamma, xi, d, scal, scale, opts, forced):
    """scale * P_m(delta J) u with the Newton recurrence of §4.2 and the
    stopping rule on the increments scale * d_m q_m; (value, m) or (None, m)."""
    q = u.copy()
    P = d[0] * q
    errs = []
    for m in range(1, opts.m_max + 1):
        q = (delta * (J @ q) - c * q) / gamma - xi[m - 1] * q
        P = P + d[m] * q
        errs.append(weighted_norm(scale * d[m] * q, scal))
        mean = float(np.mean(errs[-opts.avg_window:]))
        if forced is not None:
            if m == forced:
                return scale * P, m
            continue
        if 10.0**opts.p_order * mean < 1.0:
            return scale * P, m
    return None, opts.m_max


def phi12_leja(J, v, w, tau: float, y_inf: float, opts: LejaOptions | None = None) -> Phi12Result:
    """tau phi_1(tau J) v + tau^2 phi_2(tau J) w (see the module docstring);
    opts.replay, if given, is [s, m_1..m_s, m_phi2]."""
    opts = opts or LejaOptions()
    J = sp.csr_matrix(J)
    v = np.asarray(v, np.float64).reshape(-1)
    w = np.asarray(w, np.float64).reshape(-1)
    alpha, beta = gershgorin_interval(J, tau)
    c, gamma = focal_map(alpha, beta)
    scal = opts.tol_a + opts.tol_r * y_inf
    rep = opts.replay
    m_cap = opts.m_max if rep is None else max(opts.m_max, max(rep[1:]))
    xi = cached_leja_points(m_cap, opts.points)
    attempts = [rep[0]] if rep is not None else [2**k for k in range(opts.max_doublings + 1)]
    for s in attempts:
        delta = tau / s
        d1 = phi1_divided_differences(xi[: m_cap + 1], c / s, gamma / s)
        d2 = phi2_divided_differences(xi[: m_cap + 1], c / s, gamma / s)
        forced2 = rep[1 + s] if rep is not None else None
        o2 = LejaOptions(**{**opts.__dict__, "m_max": max(forced2, 1)}) if forced2 else opts
        inc2, m2 = _newton(J, w, delta, c / s, gamma / s, xi, d2, scal, delta * delta, o2, forced2)
        if inc2 is None:
            continue
        y = np.zeros_like(v)
        degrees = []
        ok = True
        for k in range(s):
            u = v if k == 0 else J @ y + v + (k * delta) * w
            forced = rep[1 + k] if rep is not None else None
            o = LejaOptions(**{**opts.__dict__, "m_max": max(forced, 1)}) if forced else opts
            inc, m = _newton(J, u, delta, c / s, gamma / s, xi, d1, scal, delta, o, forced)
            if inc is None:
                ok = False
                break
            degrees.append(m)
            y = y + inc + inc2
        if ok:
            return Phi12Result(y, s, degrees, m2, True)
    return Phi12Result(np.full_like(v, np.nan), attempts[-1], [], 0, False)


def erem_step_forced(prob, T, tau: float, T_in: float, T_in_rate: float, opts=None):
    """One non-autonomous EREM step (eq. ``nEERMg``) of the heat problem whose
    inflow temperature is T_in at t_n and changes at the rate T_in_rate;
    ``prob`` is the oracle HeatProblem (its physics' T_inflow is replaced by
    T_in).  Returns (T^{n+1}, Phi12Result)."""
    from dataclasses import replace

    from .timestep import HeatProblem

    T = np.asarray(T, np.float64).reshape(-1)
    ph = replace(prob.phys, T_inflow=T_in)
    pb = HeatProblem(prob.grid, ph, prob.phi, prob.lam, prob.fluxes)
    G = pb.G(T)
    J = pb.J(T)
    w = T_in_rate * inflow_sensitivity(pb.grid, ph, pb.phi, pb.lam, pb.fluxes, T_in)
    res = phi12_leja(J, G, w, tau, float(np.max(np.abs(T))), opts)
    return T + res.value, res

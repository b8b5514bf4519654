"""Time integrators of §3.2 of arXiv 1209.5553 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* EREM (eq. ``EERM``): T^{n+1} = T^n + tau phi_1(tau J_n) G(T^n, p^n), with
  J_n = D_T G(T^n, p^n) and phi_1 from real Leja interpolation (§4.2).
* ROSM(gamma) (eq. ``ROS``): T^{n+1} = T^n + tau (I - tau gamma J_n)^{-1} G(T^n).
* ROS3p (Table ``ros3``), the same form with three stages.
* ROS2(1) (eq. ``ROSMh`` with the coefficients of Table ``ros2``), autonomous
  form: (I/(tau gamma) - J) k_i = G(T + sum_{j<i} a_ij k_j) - sum_{j<i} c_ij/tau k_j,
  T^{n+1} = T^n + sum_i b_i k_i.  The diagonal c_ii of the printed table do
  not enter the sums over j < i; the D_t f terms vanish (autonomous problem).

Linear systems are solved directly (sparse LU), so the oracle's stage values
are exact up to the conditioning of the stage matrix.
* The sequential (Trotter) coupling of §3.2: pressure at T^n, then Darcy fluxes,
  then one heat step; :func:`sequential_step`.  The Strang alternative of
  §3.2 (heat tau/2, pressure, heat tau/2): :func:`strang_step`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fv
from .leja import LejaOptions, LejaResult, phi1_leja


@dataclass
class HeatProblem:
    """Everything G and J need apart from T: grid, physics, porosity,
    conductivity and the Darcy face fluxes of the current pressure."""

    grid: fv.Grid
    phys: fv.Physics
    phi: np.ndarray
    lam: np.ndarray
    fluxes: tuple

    def G(self, T):
        return fv.heat_rhs(self.grid, self.phys, self.phi, self.lam, T, self.fluxes)

    def J(self, T):
        return fv.heat_jacobian(self.grid, self.phys, self.phi, self.lam, T, self.fluxes)


def heat_problem(grid, phys, lnk, phi, lam, p, T_for_viscosity=None):
    """HeatProblem whose fluxes come from pressure p (Darcy mobility at
    ``T_for_viscosity`` when the fluid laws depend on T)."""
    fluxes = fv.darcy_fluxes(grid, phys, lnk, p, T_for_viscosity)
    return HeatProblem(grid, phys, np.asarray(phi, np.float64).reshape(-1),
                       np.asarray(lam, np.float64).reshape(-1), fluxes)


def erem_step_krylov(prob: HeatProblem, T, tau: float, opts=None):
    """One EREM step (eq. ``EERM``) with phi_1 by the Krylov substeps of
    ``oracle.krylov`` (§4.1); returns (T^{n+1}, KrylovResult)."""
    from .krylov import phi1_krylov

    T = np.asarray(T, np.float64).reshape(-1)
    res = phi1_krylov(prob.J(T), prob.G(T), tau, float(np.max(np.abs(T))), opts)
    return T + res.value, res


def erem_step(prob: HeatProblem, T, tau: float, opts: LejaOptions | None = None):
    """One EREM step (eq. ``EERM``); returns (T^{n+1}, LejaResult)."""
    T = np.asarray(T, np.float64).reshape(-1)
    G = prob.G(T)
    J = prob.J(T)
    res: LejaResult = phi1_leja(J, G, tau, float(np.max(np.abs(T))), opts)
    return T + res.value, res


# ROS2(1) coefficients (Table ros2): gamma = 1 + 1/sqrt(2), and the remaining
# entries are the fractions of gamma the table's decimals represent.
ROS2_GAMMA = 1.0 + 1.0 / math.sqrt(2.0)
ROS2_A21 = 1.0 / ROS2_GAMMA
ROS2_C21 = 2.0 / ROS2_GAMMA
ROS2_B = (3.0 / (2.0 * ROS2_GAMMA), 1.0 / (2.0 * ROS2_GAMMA))
ROS2_BHAT = (1.0 / ROS2_GAMMA, 0.0)


# ROS3p coefficients (Table ros3): gamma = (3 + sqrt 3)/6; a21 = a31 = 1/gamma,
# a32 = 0; c21 = 1/gamma^2, c31 = 2 sqrt 3, c32 = sqrt 3; b = (2, 1/sqrt 3,
# 1 - 1/sqrt 3).  The embedded weights are taken as printed.
ROS3P_GAMMA = (3.0 + math.sqrt(3.0)) / 6.0
ROS3P_A = ((1.0 / ROS3P_GAMMA,), (1.0 / ROS3P_GAMMA, 0.0))            # a21; a31, a32
ROS3P_C = ((1.0 / ROS3P_GAMMA**2,), (2.0 * math.sqrt(3.0), math.sqrt(3.0)))  # c21; c31, c32
ROS3P_B = (2.0, 1.0 / math.sqrt(3.0), 1.0 - 1.0 / math.sqrt(3.0))
ROS3P_BHAT = (2.113248654051871, 1.0, 0.4226497308103742)


def stage_matrix(J, tau: float, gamma: float):
    """I / (tau gamma) - J, the matrix of every Rosenbrock stage."""
    n = J.shape[0]
    return (sp.identity(n, format="csr") / (tau * gamma) - J).tocsc()


def rosm_step(prob: HeatProblem, T, tau: float, gamma: float):
    """ROSM(gamma), eq. ``ROS``: T + tau (I - tau gamma J)^{-1} G(T)."""
    T = np.asarray(T, np.float64).reshape(-1)
    J = prob.J(T)
    rhs = tau * prob.G(T)
    A = (sp.identity(T.size, format="csr") - tau * gamma * J).tocsc()
    return T + spla.spsolve(A, rhs)


def ros3p_step(prob: HeatProblem, T, tau: float, embedded: bool = False):
    """ROS3p step (eq. ``ROSMh``, Table ``ros3``, autonomous form as for
    ROS2(1)); with ``embedded`` also returns the second-order solution."""
    T = np.asarray(T, np.float64).reshape(-1)
    J = prob.J(T)
    lu = spla.splu(stage_matrix(J, tau, ROS3P_GAMMA))
    k = [lu.solve(prob.G(T))]
    for i in (1, 2):
        Y = T + sum(a * kj for a, kj in zip(ROS3P_A[i - 1], k))
        rhs = prob.G(Y) - sum((c / tau) * kj for c, kj in zip(ROS3P_C[i - 1], k))
        k.append(lu.solve(rhs))
    y = T + sum(b * ki for b, ki in zip(ROS3P_B, k))
    if embedded:
        return y, T + sum(b * ki for b, ki in zip(ROS3P_BHAT, k))
    return y


@dataclass
class AdaptiveResult:
    T: np.ndarray
    dts: list            # accepted step lengths
    rejected: int
    errs: list           # scaled error of every attempt, in order


def ros_integrate(prob: HeatProblem, T, t_end: float, dt0: float, scheme: str = "ros3p",
                  tol_a: float = 1e-6, tol_r: float = 1e-6, max_steps: int = 100000):
    """Adaptive Rosenbrock integration over [0, t_end] with the embedded
    solution of eq. ``ROSMh`` and the standard error control and step-size
    prediction (the paper points to Hairer and Wanner): err = RMS(y - y_hat)
    / (tol_a + tol_r ||T^n||_inf) (the uniform scale of §4.2); a step is
    accepted when err <= 1; the next length is dt min(facmax, max(0.2,
    0.9 err^(-1/p))), p the order of the scheme (2 for ROS2(1), 3 for ROS3p),
    with facmax = 5, or 1 right after a rejection; the last step ends at
    t_end.  ``prob`` is a HeatProblem or a function of T^n giving the
    problem of that step (fluid laws that depend on T re-evaluated per step).

    For the linear heat model the ROS3p difference y - y_hat vanishes
    identically: there the second stage is (1 - 1/gamma) k_1 and the printed
    b - b_hat annihilates that combination, so only nonlinear terms give
    ROS3p an error estimate."""
    step = {"ros2": ros2_step, "ros3p": ros3p_step}[scheme]
    prob_of = prob if callable(prob) else (lambda _T: prob)
    p = {"ros2": 2, "ros3p": 3}[scheme]
    T = np.asarray(T, np.float64).reshape(-1).copy()
    t, dt, facmax = 0.0, dt0, 5.0
    dts, errs, rejected = [], [], 0
    while t < t_end and len(dts) + rejected < max_steps:
        h = min(dt, t_end - t)
        y, yh = step(prob_of(T), T, h, embedded=True)
        sc = tol_a + tol_r * float(np.max(np.abs(T)))
        err = float(np.sqrt(np.mean((y - yh) ** 2))) / sc
        errs.append(err)
        pred = math.inf if err == 0.0 else 0.9 * err ** (-1.0 / p)
        if err <= 1.0:
            T = y
            t = t_end if h == t_end - t else t + h
            dts.append(h)
            grow = min(facmax, max(0.2, pred))
            facmax = 5.0
        else:
            rejected += 1
            grow = min(1.0, max(0.2, pred))
            facmax = 1.0
        dt = h * grow
    return AdaptiveResult(T, dts, rejected, errs)


def ros2_step(prob: HeatProblem, T, tau: float, embedded: bool = False):
    """ROS2(1) step; with ``embedded`` also returns the first-order solution."""
    T = np.asarray(T, np.float64).reshape(-1)
    J = prob.J(T)
    A = stage_matrix(J, tau, ROS2_GAMMA)
    lu = spla.splu(A)
    k1 = lu.solve(prob.G(T))
    k2 = lu.solve(prob.G(T + ROS2_A21 * k1) - (ROS2_C21 / tau) * k1)
    y = T + ROS2_B[0] * k1 + ROS2_B[1] * k2
    if embedded:
        return y, T + ROS2_BHAT[0] * k1 + ROS2_BHAT[1] * k2
    return y


def pressure_solve_direct(grid, phys, lnk, T=None):
    """Steady pressure by a sparse direct solve of the TPFA system."""
    A, b = fv.pressure_system(grid, phys, lnk, T)
    return spla.spsolve(A.tocsc(), b)


def pressure_solve_cg(grid, phys, lnk, T=None, p0=None, tol=1e-13, maxit=100000):
    """Steady pressure by Jacobi-preconditioned conjugate gradients, stopped
    when ||b - A p||_2 <= tol ||b||_2 (recursive residual).  Returns
    (p, iterations, relative residual)."""
    A, b = fv.pressure_system(grid, phys, lnk, T)
    x = fv.linear_head_guess(grid, phys) if p0 is None else np.array(p0, np.float64)
    dinv = 1.0 / A.diagonal()
    r = b - A @ x
    bn = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * bn:
        return x, 0, float(np.linalg.norm(r) / bn)
    z = dinv * r
    d = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ad = A @ d
        a = rz / (d @ Ad)
        x = x + a * d
        r = r - a * Ad
        rn = np.linalg.norm(r)
        if rn <= tol * bn:
            return x, it, float(rn / bn)
        z = dinv * r
        rz_new = r @ z
        d = z + (rz_new / rz) * d
        rz = rz_new
    return x, maxit, float(np.linalg.norm(r) / bn)


def strang_step(grid, phys, lnk, phi, lam, T, p, tau, opts=(None, None), pressure="direct",
                T_p=None):
    """One Strang step of §3.2 with the steady pressure of this build: an
    EREM heat step of tau/2 with the Darcy fluxes of the last pressure
    solve, the steady pressure at the new T, then a second heat step of tau/2
    with the fluxes of that pressure.  The flow subproblem hands the heat
    subproblem a velocity field, so the first half takes p with the viscosity
    at T_p, the temperature p was solved at (the previous step's half-step
    temperature; T_p = T for the first step, where p is the steady pressure at
    T^0): those fluxes are divergence-free, while re-evaluating the viscosity
    at T would not be.  Returns (T^{n+1}, p^{n+1}, T_h, (result of each
    half)), T_h the temperature p^{n+1} was solved at (the next step's T_p)."""
    prob = heat_problem(grid, phys, lnk, phi, lam, p, T if T_p is None else T_p)
    Th, r1 = erem_step(prob, T, tau / 2, opts[0])
    if pressure == "direct":
        p1 = pressure_solve_direct(grid, phys, lnk, Th)
    else:
        p1 = pressure_solve_cg(grid, phys, lnk, Th, p0=p)[0]
    prob = heat_problem(grid, phys, lnk, phi, lam, p1, Th)
    T1, r2 = erem_step(prob, Th, tau / 2, opts[1])
    return T1, p1, Th, (r1, r2)


def sequential_step(grid, phys, lnk, phi, lam, T, p_prev, tau, scheme="erem", opts=None,
                    pressure="direct"):
    """One step of the sequential (Trotter) approach of §3.2: steady pressure
    at T^n, Darcy fluxes at T^n, then one heat step of the chosen scheme.
    Returns (T^{n+1}, p^n, info)."""
    if pressure == "direct":
        p = pressure_solve_direct(grid, phys, lnk, T)
    else:
        p = pressure_solve_cg(grid, phys, lnk, T, p0=p_prev)[0]
    prob = heat_problem(grid, phys, lnk, phi, lam, p, T)
    if scheme == "erem":
        Tn, res = erem_step(prob, T, tau, opts)
        return Tn, p, res
    if scheme == "ros2":
        return ros2_step(prob, T, tau), p, None
    if scheme == "rosm1":
        return rosm_step(prob, T, tau, 1.0), p, None
    if scheme == "rosm_half":
        return rosm_step(prob, T, tau, 0.5), p, None
    raise ValueError(scheme)

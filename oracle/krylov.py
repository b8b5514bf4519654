"""Krylov (Arnoldi) approximation of phi_1 (oracle), §4.1 of arXiv 1209.5553.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The steps, in the paper's order and notation:

1. Arnoldi's algorithm (Algorithm ``alg:al2``): v_1 = v / ||v||_2; for
   j = 1..m, w = J v_j, then for i = 1..j (modified Gram-Schmidt)
   h_ij = w^T v_i, w = w - h_ij v_i; h_{j+1,j} = ||w||_2, v_{j+1} = w / h_{j+1,j}.
2. The approximation of eq. ``approphi``:
   phi_1(tau J) v ~ ||v||_2 V_{m+1} phi_1(tau Hbar_{m+1}) e_1, where Hbar_{m+1}
   is H_m bordered by the row (0, .., 0, h_{m+1,m}) and a zero column, and
   phi_1(tau Hbar_{m+1}) e_1 is read off the exponential of the augmented
   matrix [[tau Hbar_{m+1}, e_1], [0, 0]] (its last column, §4.1).
3. Local error estimate and subdivision of the step: the paper takes them from
   the truncation error of eq. ``approphi`` (the expansion it is the first two
   terms of) and leaves the rule to the cited implementation.

Readings taken here (the paper is silent on the details of step 3):

* The step is split into substeps of the linear problem y' = J y + v,
  y(0) = 0, whose solution at tau is tau phi_1(tau J) v: a substep of length
  delta from y adds delta phi_1(delta J)(J y + v), exact in exact arithmetic.
  Every substep builds its own Krylov basis from r = J y + v.
* In that expansion the term after the two that eq. ``approphi`` keeps is
  ||r|| h_{m+1,m} delta^3 (e_m^T phi_3(delta H_m) e_1) J v_{m+1}.  With
  p1 = ||r|| h_{m+1,m} delta^2 |e_m^T phi_2(delta H_m) e_1| (the size of the
  second kept term) and p2 = ||r|| h_{m+1,m} delta^3 |e_m^T phi_3(delta H_m)
  e_1| ||J v_{m+1}|| (the size of the first dropped one), the local error is
  p2 when p1 > 10 p2, p1 p2 / (p1 - p2) when p1 > p2 (a geometric tail) and p1
  otherwise; phi_2 and phi_3 of delta H_m come from the exponential of H_m
  augmented by e_1 and a shift chain.
* A substep is accepted when its error is at most 1.2 tol delta / tau, with
  the absolute tolerance tol = (tol_a + tol_r ||T^n||_inf) sqrt(N) (the 2-norm
  counterpart of the weighted RMS scale of the Leja test, §4.2); otherwise,
  and for the next substep, delta becomes 0.9 delta (tol delta / (tau err))^(1/m)
  (the error of an m-dimensional Krylov step grows like delta^(m+1)).  The
  first substep tries the whole step.
* A breakdown (h_{j+1,j} <= 1e-12 ||J||_inf) means the subspace is invariant:
  the approximation is exact and the rest of the step is taken at once.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .leja import expm_taylor

GAMMA = 0.9    # safety factor of the step-size rule
DELTA = 1.2    # accepted error, as a multiple of the tolerance share
BREAKDOWN = 1e-12


@dataclass
class KrylovOptions:
    tol_a: float = 1e-6
    tol_r: float = 1e-6
    m: int = 10                 # Krylov dimension (§5)
    max_substeps: int = 1000
    max_rejections: int = 50
    replay: list | None = None  # forced substep lengths (absolute), taken in order


@dataclass
class KrylovResult:
    value: np.ndarray           # tau phi_1(tau J) v
    substeps: list = field(default_factory=list)   # accepted substep lengths delta
    errors: list = field(default_factory=list)     # local error estimates
    rejections: int = 0
    dims: list = field(default_factory=list)       # Krylov dimension per substep


def arnoldi_mgs(J, r, m: int, breakdown: float):
    """Algorithm ``alg:al2`` on J from r: returns (beta, V, H, k) with V of
    shape (n, k+1) (the last column only when no breakdown), H of shape
    (k+1, k) and k <= m the dimension reached."""
    n = r.size
    beta = float(np.linalg.norm(r))
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = r / beta
    for j in range(m):
        w = J @ V[:, j]
        for i in range(j + 1):
            H[i, j] = float(w @ V[:, i])
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = float(np.linalg.norm(w))
        if H[j + 1, j] <= breakdown:
            return beta, V[:, : j + 1], H[: j + 2, : j + 1], j + 1, True
        V[:, j + 1] = w / H[j + 1, j]
    return beta, V, H, m, False


def phi1_hbar_e1(H, delta: float) -> np.ndarray:
    """phi_1(delta Hbar_{k+1}) e_1 from the exponential of the augmented
    matrix [[delta Hbar, e_1], [0, 0]] (eq. ``approphi``)."""
    k = H.shape[1]
    Hbar = np.zeros((k + 1, k + 1))
    Hbar[:, :k] = H[: k + 1, :k]
    A = np.zeros((k + 2, k + 2))
    A[: k + 1, : k + 1] = delta * Hbar
    A[0, k + 1] = 1.0
    return expm_taylor(A)[: k + 1, k + 1].copy()


def phi_k_e1(Hm, delta: float, kmax: int = 3):
    """[phi_1, .., phi_kmax](delta H_m) e_1 as columns: the exponential of
    [[delta H_m, e_1, 0..], [0, 0, 1, 0..], .., [0 .. 0]] holds phi_j(delta H_m)
    e_1 in column m + j."""
    m = Hm.shape[0]
    A = np.zeros((m + kmax, m + kmax))
    A[:m, :m] = delta * Hm
    A[0, m] = 1.0
    for j in range(1, kmax):
        A[m + j - 1, m + j] = 1.0
    E = expm_taylor(A)
    return E[:m, m: m + kmax]


def local_error(beta, h_next, delta, phis, avnorm):
    """Error of one substep from the expansion terms (see the readings)."""
    p1 = beta * h_next * delta**2 * abs(phis[-1, 1])
    p2 = beta * h_next * delta**3 * abs(phis[-1, 2]) * avnorm
    if p1 > 10.0 * p2:
        return p2
    if p1 > p2:
        return p1 * p2 / (p1 - p2)
    return p1


def phi1_krylov(J, v, tau: float, y_inf: float, opts: KrylovOptions | None = None) -> KrylovResult:
    """tau phi_1(tau J) v by Krylov substeps (see the module docstring)."""
    opts = opts or KrylovOptions()
    J = sp.csr_matrix(J)
    v = np.asarray(v, np.float64).reshape(-1)
    n = v.size
    m = min(opts.m, n)
    jnorm = float(np.max(np.asarray(abs(J).sum(axis=1)).reshape(-1))) if n else 0.0
    breakdown = BREAKDOWN * max(jnorm, 1e-300)
    tol = (opts.tol_a + opts.tol_r * y_inf) * np.sqrt(n)
    y = np.zeros(n)
    res = KrylovResult(value=y)
    t = 0.0
    delta = tau
    forced = list(opts.replay) if opts.replay is not None else None
    while (t < tau * (1.0 - 1e-15)) if forced is None else (len(res.substeps) < len(forced)):
        if len(res.substeps) >= opts.max_substeps:
            raise RuntimeError("Krylov: too many substeps")
        r = J @ y + v
        if not np.any(r):
            break
        beta, V, H, k, happy = arnoldi_mgs(J, r, m, breakdown)
        avnorm = 0.0 if happy else float(np.linalg.norm(J @ V[:, k]))
        if forced is not None:
            delta = float(forced[len(res.substeps)])
        else:
            delta = min(delta, tau - t)
        rej = 0
        while True:
            phis = phi_k_e1(H[:k, :k], delta)
            err = 0.0 if happy else local_error(beta, H[k, k - 1], delta, phis, avnorm)
            if forced is not None or happy or err <= DELTA * tol * delta / tau:
                break
            rej += 1
            if rej > opts.max_rejections:
                raise RuntimeError("Krylov: too many rejections")
            delta = GAMMA * delta * (tol * delta / (tau * err)) ** (1.0 / k)
        # the accepted substep: beta V_{k+1} delta phi_1(delta Hbar_{k+1}) e_1
        coef = delta * beta * phi1_hbar_e1(H[: k + 1, :k], delta)
        y = y + V[:, : coef.size] @ coef if not happy else y + V @ coef[:k]
        res.substeps.append(delta)
        res.errors.append(err)
        res.rejections += rej
        res.dims.append(k)
        t += delta
        if happy or err == 0.0:
            delta = tau - t
        else:
            delta = GAMMA * delta * (tol * delta / (tau * err)) ** (1.0 / k)
    res.value = y
    return res

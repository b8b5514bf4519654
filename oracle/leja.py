"""Real Leja point interpolation of phi_1 (oracle), §4.2 of arXiv 1209.5553.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The steps, in the paper's order and notation:

1. Spectral focal interval [alpha, beta] of tau J from Gershgorin's circle
   theorem (§4.2); the interval is mapped onto [-2, 2] by
   z = c + gamma xi with c = (alpha + beta)/2, gamma = (beta - alpha)/4.
2. Leja points on [-2, 2] (eq. ``lejaa``): xi_0 = 2 (the image of beta) and
   xi_j maximises prod_{k<j} |xi - xi_k| over the interval.
3. Divided differences d_0..d_m of phi_1(c + gamma xi) at the points: the first
   column of the matrix function phi_1(c I + gamma L_hat) with L_hat lower
   bidiagonal (points on the diagonal, ones below it), computed with a Taylor
   expansion and scaling and squaring (§4.2, not the recursion of eq. ``div``,
   which the paper warns is inaccurate).
4. Newton form (eq. ``newt``): q_0 = v, P_0 = d_0 q_0,
   q_m = ((tau J - c I)/gamma - xi_{m-1} I) q_{m-1}, P_m = P_{m-1} + d_m q_m.
5. Error estimate and stopping rule (§4.2): ||e_m|| = ||d_m q_m|| in the
   weighted norm sqrt(N^-1 sum (x_i / scal)^2), scal = tol_a + tol_r ||y^n||_inf,
   stop once 10^p times the mean of the last five estimates is below 1 (p = 2
   for EREM).  When the degree gets too large the step is split (§4.2).

Readings of the paper taken here:

* [alpha, beta] is the Gershgorin interval of tau J (the paper's L_m carries an
  extra tau_n and eq. ``newt`` writes J where tau J is meant).
* The estimate is taken on the increment tau d_m q_m that is added to the
  solution, and scal uses ||T^n||_inf as printed.
* The mean runs over e_max(1, m-4) .. e_m from m = 1 on; m_max = 150 terms.
* Splitting: when m_max terms do not meet the test, the number of substeps s
  is doubled (at most ``max_doublings`` times) and the step restarts with
  delta = tau / s; substep k adds delta phi_1(delta J)(J w_k + v) to w_k,
  which composes tau phi_1(tau J) v exactly in exact arithmetic.
* Ties in the Leja maximisation (only at j = 3, by symmetry) go to the
  smaller point.
* When beta - alpha is zero (a single cell, or J a multiple of I) the
  interval is widened so that gamma >= 1e-8 max(1, |c|).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# step 1: Gershgorin interval
# --------------------------------------------------------------------------
def gershgorin_interval(J, tau: float):
    """[alpha, beta] containing the spectrum of tau J (Gershgorin circles,
    which for a real matrix meet the real axis in [J_ii - R_i, J_ii + R_i])."""
    J = sp.csr_matrix(J)
    diag = J.diagonal()
    radius = np.asarray(abs(J).sum(axis=1)).reshape(-1) - np.abs(diag)
    alpha = tau * np.min(diag - radius)
    beta = tau * np.max(diag + radius)
    return float(alpha), float(beta)


GAMMA_FLOOR = 1e-8


def focal_map(alpha: float, beta: float):
    """c and gamma of the map xi -> c + gamma xi from [-2, 2] onto [alpha, beta]."""
    c = 0.5 * (alpha + beta)
    gamma = 0.25 * (beta - alpha)
    gamma = max(gamma, GAMMA_FLOOR * max(1.0, abs(c)))
    return c, gamma


# --------------------------------------------------------------------------
# step 2: Leja points on [-2, 2]
# --------------------------------------------------------------------------
def _log_product(x, pts):
    return float(np.sum(np.log(np.abs(x - pts))))


def _gap_maximiser(a, b, pts):
    """Maximiser of sum_k log|x - pts_k| inside the gap (a, b) between two
    consecutive points.  The function is concave there, so its maximiser is
    the single zero of the derivative sum_k 1/(x - pts_k), which falls from
    +inf at a to -inf at b; bisection finds it to the last bit."""
    lo, hi = a, b
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if np.sum(1.0 / (mid - pts)) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def leja_points(M: int, tie_tol: float = 1e-12) -> np.ndarray:
    """xi_0 .. xi_M on [-2, 2] from eq. ``lejaa`` with xi_0 = 2."""
    pts = [2.0]
    for _ in range(M):
        P = np.array(pts)
        cands = []
        if -2.0 not in pts:
            cands.append(-2.0)  # product is largest at the far end
        s = np.sort(P)
        for a, b in zip(s[:-1], s[1:]):
            cands.append(_gap_maximiser(a, b, P))
        vals = [_log_product(x, P) for x in cands]
        best = max(vals)
        ties = [x for x, v in zip(cands, vals) if v >= best - tie_tol * max(1.0, abs(best))]
        pts.append(min(ties))
    return np.array(pts)


def fast_leja_points(M: int, tie_tol: float = 1e-12) -> np.ndarray:
    """The fast variant of eq. ``lejaa`` (the "real fast Leja" name of §4.2;
    the candidate rule of Baglama, Calvetti and Reichel): xi_0 = 2, xi_1 = -2,
    and every later point is, among the midpoints of the gaps between
    consecutive points chosen so far, the one where prod_k |xi - xi_k| is
    largest (ties to the smaller point).  The maximisation of eq. ``lejaa``
    over the whole interval becomes one over a finite candidate set."""
    pts = [2.0]
    if M >= 1:
        pts.append(-2.0)
    while len(pts) < M + 1:
        P = np.array(pts)
        s = np.sort(P)
        cands = 0.5 * (s[:-1] + s[1:])
        vals = [_log_product(x, P) for x in cands]
        best = max(vals)
        ties = [x for x, v in zip(cands, vals) if v >= best - tie_tol * max(1.0, abs(best))]
        pts.append(float(min(ties)))
    return np.array(pts[: M + 1])


# --------------------------------------------------------------------------
# step 3: divided differences by the matrix function
# --------------------------------------------------------------------------
def expm_taylor(A, degree: int | None = None, target: float = 0.5):
    """exp(A) by a Taylor polynomial of A / 2^s and s squarings, with s the
    smallest integer for which ||A||_1 / 2^s <= 0.5.

    The default degree is the matrix size plus 30: for the bidiagonal
    matrices of the divided differences, entry (j, 0) of A^k is zero for
    k < j, so an entry far below the diagonal only keeps its relative
    accuracy when the polynomial reaches well past power j."""
    A = np.asarray(A, dtype=np.float64)
    if degree is None:
        degree = A.shape[0] + 30
    norm = np.max(np.sum(np.abs(A), axis=0)) if A.size else 0.0
    s = 0
    while norm / 2.0**s > target:
        s += 1
    B = A / 2.0**s
    E = np.eye(A.shape[0])
    term = np.eye(A.shape[0])
    for k in range(1, degree + 1):
        term = term @ B / k
        E = E + term
    for _ in range(s):
        E = E @ E
    return E


def phi1_divided_differences(xi, c: float, gamma: float) -> np.ndarray:
    """d_j = phi_1[xi_0, ..., xi_j] of the function xi -> phi_1(c + gamma xi).

    They are the first column of phi_1(L), L = c I + gamma L_hat (§4.2).  That
    column is read off the exponential of the augmented matrix
    [[L, e_1], [0, 0]], whose upper-right column is phi_1(L) e_1 (since
    phi_1(L) = sum_k L^k / (k+1)!)."""
    xi = np.asarray(xi, np.float64)
    m1 = xi.size
    L = c * np.eye(m1) + gamma * (np.diag(xi) + np.diag(np.ones(m1 - 1), -1))
    A = np.zeros((m1 + 1, m1 + 1))
    A[:m1, :m1] = L
    A[0, m1] = 1.0
    return expm_taylor(A)[:m1, m1].copy()


# --------------------------------------------------------------------------
# steps 4-5: Newton form, error estimate, substeps
# --------------------------------------------------------------------------
@dataclass
class LejaOptions:
    tol_a: float = 1e-6
    tol_r: float = 1e-6
    p_order: int = 2
    m_max: int = 150
    max_doublings: int = 6
    avg_window: int = 5
    replay: list | None = None  # [s, m_1, ..., m_s]
    points: str = "exact"       # "exact" (eq. lejaa) or "fast" (midpoint candidates)
    # substep count the first attempt takes (a power of two; the doubling on
    # failure goes on from there up to 2**max_doublings).  §4.2 fixes only the
    # doubling: 1 restarts every step from one substep, the last step's count
    # continues where it stopped.
    start_substeps: int = 1


@dataclass
class LejaResult:
    value: np.ndarray  # tau phi_1(tau J) v
    substeps: int
    degrees: list = field(default_factory=list)
    alpha: float = 0.0
    beta: float = 0.0
    err_est: float = 0.0
    converged: bool = True

    @property
    def schedule(self):
        return [self.substeps] + list(self.degrees)


_LEJA_CACHE: dict[tuple, np.ndarray] = {}


def cached_leja_points(M: int, points: str = "exact") -> np.ndarray:
    make = {"exact": leja_points, "fast": fast_leja_points}[points]
    best = max((k for (kind, k) in _LEJA_CACHE if kind == points and k >= M), default=None)
    if best is None:
        _LEJA_CACHE[(points, M)] = make(M)
        best = M
    return _LEJA_CACHE[(points, best)][: M + 1]


def weighted_norm(x, scal):
    """The weighted, scaled norm of §4.2: sqrt(N^-1 sum (x_i / scal_i)^2)."""
    return float(np.sqrt(np.mean((x / scal) ** 2)))


def _newton_leja_substep(J, u, delta, c, gamma, xi, d, scal, opts, forced_degree):
    """One interpolation of delta phi_1(delta J) u; returns (delta * P_m, m, err).

    c, gamma describe the interval of delta J.  With ``forced_degree`` the
    stopping rule is not applied and exactly that many terms are taken."""
    q = u.copy()
    P = d[0] * q
    errs = []
    for m in range(1, opts.m_max + 1):
        q = (delta * (J @ q) - c * q) / gamma - xi[m - 1] * q
        P = P + d[m] * q
        errs.append(weighted_norm(delta * d[m] * q, scal))
        mean = float(np.mean(errs[-opts.avg_window:]))
        if forced_degree is not None:
            if m == forced_degree:
                return delta * P, m, mean
            continue
        if 10.0**opts.p_order * mean < 1.0:
            return delta * P, m, mean
    return None, opts.m_max, float(np.mean(errs[-opts.avg_window:]))


def phi1_leja(J, v, tau: float, y_inf: float, opts: LejaOptions | None = None) -> LejaResult:
    """tau phi_1(tau J) v by real Leja interpolation with the stopping rule and
    substep doubling described in the module docstring."""
    opts = opts or LejaOptions()
    J = sp.csr_matrix(J)
    v = np.asarray(v, np.float64).reshape(-1)
    alpha, beta = gershgorin_interval(J, tau)
    c, gamma = focal_map(alpha, beta)
    scal = opts.tol_a + opts.tol_r * y_inf
    m_cap = opts.m_max
    if opts.replay is not None:
        m_cap = max(m_cap, max(opts.replay[1:]))
    xi = cached_leja_points(m_cap, opts.points)
    first = min(max(1, opts.start_substeps), 2**opts.max_doublings)
    attempts = [opts.replay[0]] if opts.replay is not None else [
        2**k for k in range(opts.max_doublings + 1) if 2**k >= first]
    last_err = 0.0
    for s in attempts:
        delta = tau / s
        d = phi1_divided_differences(xi[: m_cap + 1], c / s, gamma / s)
        w = np.zeros_like(v)
        degrees = []
        ok = True
        for k in range(s):
            u = v if k == 0 else J @ w + v
            forced = opts.replay[1 + k] if opts.replay is not None else None
            if forced is not None:
                o = LejaOptions(**{**opts.__dict__, "m_max": max(forced, 1)})
            else:
                o = opts
            inc, m, last_err = _newton_leja_substep(J, u, delta, c / s, gamma / s, xi, d, scal, o, forced)
            if inc is None:
                ok = False
                break
            degrees.append(m)
            w = w + inc
        if ok:
            return LejaResult(w, s, degrees, alpha, beta, last_err, True)
    return LejaResult(np.full_like(v, np.nan), attempts[-1], [], alpha, beta, last_err, False)

"""Pins of the oracle's Leja machinery (§4.2) against things other than itself:
closed forms, brute force, high-precision arithmetic and dense matrix
exponentials."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fv, leja
from oracle.leja import LejaOptions


def test_first_leja_points_closed_form():
    # xi_0 = 2; |xi - 2| is largest at -2; |xi^2 - 4| at 0; |xi (xi^2 - 4)| at
    # +-2/sqrt(3) (equal products, the tie goes to the smaller point).
    xi = leja.leja_points(3)
    assert xi[0] == 2.0 and xi[1] == -2.0
    assert abs(xi[2]) < 1e-15
    assert xi[3] == pytest.approx(-2.0 / math.sqrt(3.0), abs=1e-15)


def test_leja_points_brute_force():
    # every new point maximises prod |xi - xi_k| on a 2e6-point grid
    xi = leja.leja_points(24)
    grid = np.linspace(-2.0, 2.0, 2_000_001)
    step = grid[1] - grid[0]
    for j in range(1, 25):
        logp = np.zeros_like(grid)
        for k in range(j):
            with np.errstate(divide="ignore"):
                logp += np.log(np.abs(grid - xi[k]))
        best = grid[np.argmax(logp)]
        if j == 3:
            continue  # symmetric tie, checked above
        assert abs(best - xi[j]) <= 2 * step, (j, best, xi[j])


def test_leja_points_distinct_bounded_and_capacity():
    xi = leja.leja_points(150)
    assert np.all(np.abs(xi) <= 2.0)
    assert len(np.unique(xi)) == xi.size
    # (prod_{k<j} |xi_j - xi_k|)^(1/j) tends to the capacity of [-2, 2], which is 1
    j = 150
    g = np.exp(np.mean(np.log(np.abs(xi[j] - xi[:j]))))
    assert 0.9 < g < 1.6


def _mp_divided_differences(xi, c, gamma, mp):
    xs = [mp.mpf(float(x)) for x in xi]

    def phi1(z):
        return mp.expm1(z) / z if z != 0 else mp.mpf(1)

    col = [phi1(mp.mpf(c) + mp.mpf(gamma) * x) for x in xs]
    out = [col[0]]
    for j in range(1, len(xs)):
        col = [(col[i + 1] - col[i]) / (xs[i + j] - xs[i]) for i in range(len(col) - 1)]
        out.append(col[0])
    return out


@pytest.mark.parametrize("c,gamma", [(-20.0, 10.0), (-3.0, 1.5), (-60.0, 30.0), (-0.5, 0.25), (-5.0, 5.0)])
def test_divided_differences_vs_high_precision(c, gamma):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160
    xi = leja.leja_points(45)
    d = leja.phi1_divided_differences(xi, c, gamma)
    ref = _mp_divided_differences(xi, c, gamma, mp)
    for j, r in enumerate(ref):
        r = float(r)
        if abs(r) > 1e-280:
            assert abs(d[j] - r) <= 1e-11 * abs(r), (j, d[j], r)


def test_divided_difference_zero_is_phi1_at_beta():
    xi = leja.leja_points(10)
    for c, gamma in [(-20.0, 10.0), (-1.0, 0.3)]:
        beta = c + 2 * gamma
        d = leja.phi1_divided_differences(xi, c, gamma)
        want = math.expm1(beta) / beta if beta != 0 else 1.0
        assert d[0] == pytest.approx(want, rel=1e-14)


def _small_problem(nx=7, ny=5, pe=20.0, seed=3):
    rng = np.random.default_rng(seed)
    g = fv.Grid(2, nx, ny)
    lnk = rng.normal(0, 1, g.n)
    ph = fv.Physics(rhoc_f=pe, rhoc_s=pe, T_inflow=80.0)
    from oracle.timestep import heat_problem, pressure_solve_direct

    p = pressure_solve_direct(g, ph, lnk)
    prob = heat_problem(g, ph, lnk, np.full(g.n, 0.2), rng.uniform(0.5, 2.0, g.n), p)
    T = rng.uniform(20, 80, g.n)
    return prob, T


def _phi1_expm(J, v, tau):
    n = J.shape[0]
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = tau * J.toarray()
    A[:n, n] = tau * v
    return sla.expm(A)[:n, n]


@pytest.mark.parametrize("tau", [0.01, 0.05, 0.3])
def test_phi1_leja_matches_dense_expm(tau):
    prob, T = _small_problem()
    J = prob.J(T)
    v = prob.G(T)
    ref = _phi1_expm(J, v, tau)
    res = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))), LejaOptions(tol_a=1e-13, tol_r=1e-13))
    assert res.converged
    err = np.linalg.norm(res.value - ref) / np.linalg.norm(ref)
    assert err < 1e-10, (err, res.schedule)


def test_phi1_leja_default_tolerance_bound():
    # at the paper's tolerance (1e-6) the weighted error of the increment stays
    # at the tolerance level
    prob, T = _small_problem()
    tau = 0.05
    J, v = prob.J(T), prob.G(T)
    ref = _phi1_expm(J, v, tau)
    res = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))), LejaOptions())
    scal = 1e-6 + 1e-6 * np.max(np.abs(T))
    assert leja.weighted_norm(res.value - ref, scal) < 1.0


def test_phi1_fourier_modes_periodic_advection_diffusion():
    # periodic upwind advection-diffusion on a ring: J is circulant with
    # eigenvectors exp(i k x) and eigenvalues
    # lambda_k = D (2 cos(k h) - 2)/h^2 - (u/h)(1 - exp(-i k h)).
    n, D, u, tau = 64, 0.01, 1.0, 0.02
    h = 1.0 / n
    main = np.full(n, -2 * D / h**2 - u / h)
    lower = np.full(n, D / h**2 + u / h)
    upper = np.full(n, D / h**2)
    J = sp.diags([main, lower[1:], upper[:-1]], [0, -1, 1], shape=(n, n)).tolil()
    J[0, n - 1] = lower[0]
    J[n - 1, 0] = upper[0]
    J = J.tocsr()
    x = np.arange(n) * h
    modes = [(1, 1.0), (3, 0.5), (7, -0.25)]
    v = sum(a * np.cos(2 * np.pi * k * x) for k, a in modes)
    exact = np.zeros(n, dtype=complex)
    for k, a in modes:
        th = 2 * np.pi * k * h
        lam = D * (2 * np.cos(th) - 2) / h**2 - (u / h) * (1 - np.exp(-1j * th))
        z = tau * lam
        ph1 = np.expm1(z) / z
        # cos = (e^{i} + e^{-i})/2 ; the conjugate mode has the conjugate eigenvalue
        exact += a * 0.5 * tau * (ph1 * np.exp(1j * th * np.arange(n)) + np.conj(ph1) * np.exp(-1j * th * np.arange(n)))
    exact = exact.real
    res = leja.phi1_leja(J, v, tau, 1.0, LejaOptions(tol_a=1e-12, tol_r=1e-12))
    assert res.converged
    assert np.max(np.abs(res.value - exact)) < 1e-10 * np.max(np.abs(exact))


def test_superlinear_convergence():
    prob, T = _small_problem(pe=5.0)
    tau = 0.05
    J, v = prob.J(T), prob.G(T)
    ref = _phi1_expm(J, v, tau)
    roots = []
    # the m-th root of the error falls towards 0 (§4.2); Leja points alternate
    # sides of the interval, so compare every fourth degree
    for m in (4, 8, 12, 16):
        res = leja.phi1_leja(J, v, tau, 1.0, LejaOptions(replay=[1, m]))
        err = np.linalg.norm(res.value - ref) / np.linalg.norm(ref)
        if err < 1e-12:  # rounding floor reached
            break
        roots.append(err ** (1.0 / m))
    assert len(roots) >= 3 and roots[-1] < 0.75 * roots[0]
    assert all(b < a for a, b in zip(roots, roots[1:])), roots


def test_substeps_compose_the_same_action():
    prob, T = _small_problem()
    tau = 0.2
    J, v = prob.J(T), prob.G(T)
    ref = _phi1_expm(J, v, tau)
    for s in (2, 4):
        res = leja.phi1_leja(J, v, tau, 1.0, LejaOptions(tol_a=1e-12, tol_r=1e-12,
                                                        replay=None, max_doublings=0, m_max=150))
        assert np.linalg.norm(res.value - ref) < 1e-9 * np.linalg.norm(ref)
        forced = leja.phi1_leja(J, v, tau, 1.0, LejaOptions(replay=[s] + [60] * s))
        assert np.linalg.norm(forced.value - ref) < 1e-9 * np.linalg.norm(ref)


def test_degree_cap_triggers_substep_doubling():
    prob, T = _small_problem(pe=50.0)
    tau = 0.5
    J, v = prob.J(T), prob.G(T)
    ref = _phi1_expm(J, v, tau)
    res = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))), LejaOptions(m_max=12))
    assert res.converged and res.substeps > 1
    scal = 1e-6 + 1e-6 * np.max(np.abs(T))
    assert leja.weighted_norm(res.value - ref, scal) < 10.0
    fail = leja.phi1_leja(J, v, tau, 1.0, LejaOptions(m_max=3, max_doublings=0))
    assert not fail.converged


def test_substep_start_skips_the_smaller_levels():
    # starting at s0 substeps: the attempts below s0 are not taken, the value
    # is still the phi_1 action within the tolerance, and a start at or above
    # the count the doubling reaches gives the doubling's own result
    prob, T = _small_problem(pe=50.0)
    tau = 0.5
    J, v = prob.J(T), prob.G(T)
    ref = _phi1_expm(J, v, tau)
    scal = 1e-6 + 1e-6 * np.max(np.abs(T))
    base = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))), LejaOptions(m_max=12))
    assert base.converged and base.substeps >= 2
    same = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))),
                          LejaOptions(m_max=12, start_substeps=base.substeps))
    assert same.schedule == base.schedule and np.array_equal(same.value, base.value)
    up = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))),
                        LejaOptions(m_max=12, start_substeps=2 * base.substeps))
    assert up.converged and up.substeps == 2 * base.substeps
    assert leja.weighted_norm(up.value - ref, scal) < 10.0
    capped = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))),
                            LejaOptions(m_max=40, max_doublings=1, start_substeps=64))
    assert capped.substeps == 2


def test_gershgorin_interval_contains_spectrum():
    prob, T = _small_problem()
    tau = 0.1
    J = prob.J(T)
    alpha, beta = leja.gershgorin_interval(J, tau)
    ev = np.linalg.eigvals(tau * J.toarray())
    assert np.all(ev.real >= alpha - 1e-9) and np.all(ev.real <= beta + 1e-9)


def test_stopping_settings_match_paper():
    import os

    here = os.path.join(os.path.dirname(__file__), "golden", "paper_settings.txt")
    vals = {}
    for line in open(here):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    o = LejaOptions()
    assert o.tol_a == vals["tol"] and o.tol_r == vals["tol"]
    assert o.p_order == vals["p_order"] and o.avg_window == vals["avg"]


# ---------------------------------------------------------------------------
# the fast (midpoint-candidate) Leja points, the option behind the name of §4.2
# ---------------------------------------------------------------------------
def test_first_fast_leja_points_closed_form():
    # 2, -2; the only gap midpoint is 0; then -1 and 1 tie (product 3: the
    # smaller wins) and 1 follows (product 6 against 1.31 at -1.5); then
    # -1.5 and 1.5 tie at 3.28 and -0.5 follows
    assert list(leja.fast_leja_points(7)) == [2.0, -2.0, 0.0, -1.0, 1.0, -1.5, 1.5, -0.5]


def test_fast_leja_points_brute_force():
    # every new point is, over all midpoints of consecutive chosen points
    # (enumerated afresh), one with the largest product, the smallest on ties;
    # every point is a dyadic rational (a midpoint of midpoints of +-2)
    xi = leja.fast_leja_points(60)
    for j in range(2, 61):
        s = sorted(xi[:j])
        mids = [(a + b) / 2 for a, b in zip(s[:-1], s[1:])]
        prods = [math.prod(abs(m - x) for x in xi[:j]) for m in mids]
        best = max(prods)
        winners = [m for m, p in zip(mids, prods) if p >= best * (1 - 1e-12)]
        assert xi[j] == min(winners), j
        assert float(xi[j] * 2**40).is_integer()


def test_fast_leja_points_distinct_bounded_and_capacity():
    xi = leja.fast_leja_points(150)
    assert np.all(np.abs(xi) <= 2.0)
    assert len(np.unique(xi)) == xi.size
    j = 150
    g = np.exp(np.mean(np.log(np.abs(xi[j] - xi[:j]))))
    assert 0.9 < g < 1.6


@pytest.mark.parametrize("tau", [0.01, 0.05, 0.3])
def test_phi1_fast_leja_matches_dense_expm(tau):
    prob, T = _small_problem()
    J = prob.J(T)
    v = prob.G(T)
    ref = _phi1_expm(J, v, tau)
    res = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))),
                         LejaOptions(tol_a=1e-13, tol_r=1e-13, points="fast"))
    assert res.converged
    err = np.linalg.norm(res.value - ref) / np.linalg.norm(ref)
    assert err < 1e-10, (err, res.schedule)
    # the two point sets give the same function value through different
    # polynomials
    exact = leja.phi1_leja(J, v, tau, float(np.max(np.abs(T))), LejaOptions(tol_a=1e-13, tol_r=1e-13))
    assert np.linalg.norm(res.value - exact.value) / np.linalg.norm(ref) < 2e-10


# ---------------------------------------------------------------------------
# the stopping rule of §4.2, pinned on a diagonal J whose Newton vectors have a
# closed form, so the sequence of error estimates e_m is known without the
# oracle's recurrence or its divided-difference routine
# ---------------------------------------------------------------------------
def _closed_form_estimates(lam, v, tau, y_inf, tol, M, mp):
    """e_1..e_M for J = diag(lam): the interval of tau J is [tau min, tau max];
    mode i of q_m is v_i prod_{k<m} ((tau lam_i - c)/gamma - xi_k); d_m are
    160-digit recursive divided differences; e_m is the weighted RMS of the
    increment tau d_m q_m with scal = tol_a + tol_r ||y||_inf (tol_a = tol_r)."""
    alpha, beta = tau * lam.min(), tau * lam.max()
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    xi = leja.leja_points(M)
    d = [float(x) for x in _mp_divided_differences(xi, c, gamma, mp)]
    z = (tau * lam - c) / gamma
    scal = tol + tol * y_inf
    q = np.asarray(v, np.float64).copy()
    e = []
    for m in range(1, M + 1):
        q = q * (z - xi[m - 1])
        e.append(math.sqrt(float(np.mean((tau * d[m] * q / scal) ** 2))))
    return np.array(e)


def _first_stop(e, window, p=2, divisor=None, first=1):
    """First m >= first with 10^p times the mean of the last `window`
    estimates (those that exist) below 1; `divisor` replaces the count of
    averaged estimates (a zero-padded mean)."""
    for m in range(first, len(e) + 1):
        tail = e[max(0, m - window):m]
        mean = float(np.sum(tail)) / (divisor or tail.size)
        if 10.0**p * mean < 1.0:
            return m
    return None


def _diagonal_case(n, lam_max, seed):
    rng = np.random.default_rng(seed)
    lam = -np.sort(rng.uniform(0.0, lam_max, n))
    lam[0], lam[-1] = 0.0, -lam_max
    return lam, rng.normal(0.0, 1.0, n)


@pytest.mark.parametrize("n,lam_max,tau,y_inf,tol", [
    (40, 50.0, 1.0, 1.0, 1e-6),    # window 4 / 5 / 6 stop at 29 / 30 / 31
    (40, 200.0, 0.5, 80.0, 1e-8),  # tau != 1 and a state scale in scal
    (64, 400.0, 0.25, 20.0, 3e-7),
])
def test_stopping_rule_degree_from_closed_form_estimates(n, lam_max, tau, y_inf, tol):
    # §4.2: stop at the first m where 10^p (p = 2) times the mean of the last
    # five estimates is below 1.  The case is chosen so that a window of 4 or
    # 6, the last estimate alone, or a stop one term late each give another
    # degree than the rule as printed.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160
    lam, v = _diagonal_case(n, lam_max, seed=7)
    e = _closed_form_estimates(lam, v, tau, y_inf, tol, 90, mp)
    want = _first_stop(e, 5)
    assert want is not None
    variants = {_first_stop(e, 4), _first_stop(e, 6), _first_stop(e, 1), want + 1}
    assert want not in variants, (want, variants)
    res = leja.phi1_leja(sp.diags(lam), v, tau, y_inf, LejaOptions(tol_a=tol, tol_r=tol))
    assert res.converged and res.substeps == 1
    assert res.degrees == [want]
    # the reported estimate is that mean at the stopping degree
    assert res.err_est == pytest.approx(float(np.mean(e[want - 5:want])), rel=1e-9)
    # the value is the Newton sum up to that degree: tau phi_1(tau lam) v
    # within the estimate's tolerance, mode by mode
    exact = tau * np.array([math.expm1(tau * x) / (tau * x) if x != 0 else 1.0 for x in lam]) * v
    scal = tol + tol * y_inf
    assert leja.weighted_norm(res.value - exact, scal) < 1.0


def test_stopping_rule_averages_the_estimates_that_exist_at_the_start():
    # before five estimates exist the mean runs over e_1..e_m (§4.2 gives no
    # minimum degree).  v is scaled so that 10^p e_1 = 2.5 and the later
    # estimates are far smaller: the rule stops at m = 3, where the mean first
    # drops below 10^-p; a zero-padded mean (sum / 5) would stop at m = 1, a
    # rule that waits for five estimates at m = 5, the last estimate alone at
    # m = 2.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160
    lam, v = _diagonal_case(16, 0.5, seed=3)
    tol, tau = 1e-3, 1.0
    e1 = _closed_form_estimates(lam, v, tau, 1.0, tol, 1, mp)[0]
    v = v * (2.5 / (100.0 * e1))
    e = _closed_form_estimates(lam, v, tau, 1.0, tol, 20, mp)
    assert 100.0 * e[0] == pytest.approx(2.5, rel=1e-12) and 100.0 * e[1] < 0.4
    want = _first_stop(e, 5)
    assert want == 3
    assert _first_stop(e, 5, divisor=5) == 1
    assert _first_stop(e, 5, first=5) == 5
    assert _first_stop(e, 1) == 2
    res = leja.phi1_leja(sp.diags(lam), v, tau, 1.0, LejaOptions(tol_a=tol, tol_r=tol))
    assert res.degrees == [want] and res.substeps == 1

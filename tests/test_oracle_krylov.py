"""Pins of the oracle's Krylov phi_1 (oracle/krylov.py, §4.1): the Arnoldi
relation and orthonormality of Algorithm ``alg:al2``, breakdown on an
invariant subspace, phi_k of small matrices against their closed forms (via
scipy's expm and a linear solve, not the oracle's Taylor routine), exactness
once the Krylov dimension reaches N, the error against a dense matrix
exponential on small grids, and agreement with the independent Leja path."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import cases as C
from oracle import krylov as K, leja, timestep as ts


def _dense_phi1(J, v, tau):
    n = v.size
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = tau * J
    A[:n, n] = v
    return tau * sl.expm(A)[:n, n]


def _phi_closed(X, k):
    """phi_k(X) = X^{-k} (e^X - sum_{j<k} X^j / j!) for invertible X."""
    n = X.shape[0]
    acc = sl.expm(X)
    term = np.eye(n)
    for j in range(k):
        acc = acc - term
        term = term @ X / (j + 1)
    return np.linalg.solve(np.linalg.matrix_power(X, k), acc)


def test_arnoldi_relation_and_orthonormality():
    rng = np.random.default_rng(1)
    n, m = 60, 10
    J = sp.random(n, n, density=0.1, random_state=2, format="csr") - 3 * sp.identity(n)
    r = rng.standard_normal(n)
    beta, V, H, k, happy = K.arnoldi_mgs(J, r, m, 1e-14)
    assert not happy and k == m
    assert abs(beta - np.linalg.norm(r)) < 1e-12 * beta
    assert np.max(np.abs(V.T @ V - np.eye(m + 1))) < 1e-12
    lhs = J @ V[:, :m]
    assert np.max(np.abs(lhs - V @ H)) < 1e-12 * np.max(np.abs(lhs))
    # H is upper Hessenberg with positive subdiagonal
    assert np.all(np.tril(H[:m, :m], -2) == 0) and np.all(np.diag(H, -1) > 0)


def test_arnoldi_breaks_down_on_an_invariant_subspace():
    n = 30
    J = sp.diags(np.arange(1.0, n + 1))
    r = np.zeros(n)
    r[[3, 7, 20]] = [1.0, -2.0, 0.5]   # spans three eigenvectors
    beta, V, H, k, happy = K.arnoldi_mgs(J, r, 10, 1e-12 * n)
    assert happy and k == 3
    # the Ritz values are the three eigenvalues
    assert np.allclose(np.sort(np.linalg.eigvals(H[:3, :3]).real), [4.0, 8.0, 21.0], atol=1e-10)


@pytest.mark.parametrize("delta", [0.3, 2.0])
def test_phi_k_e1_match_closed_forms(delta):
    rng = np.random.default_rng(3)
    m = 8
    Hm = np.triu(rng.standard_normal((m, m)), -1) - 2 * np.eye(m)
    got = K.phi_k_e1(Hm, delta)
    for k in (1, 2, 3):
        want = _phi_closed(delta * Hm, k)[:, 0]
        assert np.max(np.abs(got[:, k - 1] - want)) < 1e-11 * max(1.0, np.max(np.abs(want)))


def test_phi1_hbar_is_phi1_of_hm_plus_the_corrector():
    # eq. approphi: the first m entries are phi_1(delta H_m) e_1, the last is
    # delta h_{m+1,m} e_m^T phi_2(delta H_m) e_1
    rng = np.random.default_rng(4)
    m, delta = 6, 0.7
    H = np.zeros((m + 1, m))
    H[:m, :m] = np.triu(rng.standard_normal((m, m)), -1) - np.eye(m)
    H[m, m - 1] = 0.37
    got = K.phi1_hbar_e1(H, delta)
    Hm = H[:m, :m]
    assert np.max(np.abs(got[:m] - _phi_closed(delta * Hm, 1)[:, 0])) < 1e-12
    corr = delta * 0.37 * _phi_closed(delta * Hm, 2)[m - 1, 0]
    assert abs(got[m] - corr) < 1e-12 * max(1.0, abs(corr))


def test_krylov_is_exact_once_the_dimension_reaches_n():
    case = C.heat2d_rect(3, 3)
    J = case.problem().J(case.T0)
    v = case.problem().G(case.T0)
    res = K.phi1_krylov(J, v, case.dt, float(np.max(case.T0)))
    want = _dense_phi1(J.toarray(), v, case.dt)
    assert res.dims[0] <= 9 and len(res.substeps) == 1
    assert np.linalg.norm(res.value - want) < 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("shape", [(16, 16), (12, 9)])
def test_krylov_meets_its_tolerance_against_a_dense_exponential(shape):
    case = C.heat2d_rect(*shape)
    pb = case.problem()
    J, v = pb.J(case.T0), pb.G(case.T0)
    yinf = float(np.max(np.abs(case.T0)))
    opts = K.KrylovOptions(tol_a=1e-6, tol_r=1e-6)
    res = K.phi1_krylov(J, v, case.dt, yinf, opts)
    want = _dense_phi1(J.toarray(), v, case.dt)
    tol = (opts.tol_a + opts.tol_r * yinf) * np.sqrt(v.size)
    assert abs(sum(res.substeps) - case.dt) < 1e-14
    assert np.linalg.norm(res.value - want) <= 2 * tol
    # the step-size rule, delta (tol delta / (tau err))^(1/m), lands within one
    # rejection of an acceptable substep
    assert res.rejections <= len(res.substeps)
    # a tighter tolerance takes more substeps and lands closer
    tight = K.phi1_krylov(J, v, case.dt, yinf, K.KrylovOptions(tol_a=1e-10, tol_r=1e-10))
    assert len(tight.substeps) > len(res.substeps)
    assert np.linalg.norm(tight.value - want) < np.linalg.norm(res.value - want)


def test_krylov_agrees_with_the_leja_path_on_the_64_grid():
    case = C.heat2d(64)
    pb = case.problem()
    J, v = pb.J(case.T0), pb.G(case.T0)
    yinf = float(np.max(np.abs(case.T0)))
    kr = K.phi1_krylov(J, v, case.dt, yinf)
    lj = leja.phi1_leja(J, v, case.dt, yinf)
    assert np.linalg.norm(kr.value - lj.value) < 1e-7 * np.linalg.norm(lj.value)


def test_replay_reproduces_the_free_run_and_erem_step():
    case = C.heat2d(32)
    pb = case.problem()
    T1, res = ts.erem_step_krylov(pb, case.T0, case.dt)
    T2, res2 = ts.erem_step_krylov(pb, case.T0, case.dt, K.KrylovOptions(replay=res.substeps))
    assert res2.substeps == res.substeps
    assert np.array_equal(T1, T2)
    T3, _ = ts.erem_step(pb, case.T0, case.dt)
    assert np.linalg.norm(T1 - T3) < 1e-7 * np.linalg.norm(T3 - case.T0)

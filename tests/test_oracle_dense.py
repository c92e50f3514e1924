"""Pins of the oracle's dense kernels against textbook definitions and LAPACK."""
import numpy as np
import pytest
import scipy.linalg as sla


def _spd(rng, n, cond=1e6):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (q * np.logspace(0, np.log10(cond), n)) @ q.T


@pytest.mark.parametrize("n", [1, 2, 7, 33, 80])
def test_cholesky_matches_numpy(oracle_lib, n):
    rng = np.random.default_rng(n)
    a = _spd(rng, n)
    g = oracle_lib.dense_chol(a)
    np.testing.assert_allclose(g, np.linalg.cholesky(a), rtol=0, atol=1e-12 * np.abs(g).max())
    assert np.all(np.triu(g, 1) == 0)


def test_cholesky_rejects_indefinite(oracle_lib):
    a = np.diag([1.0, 2.0, -1.0, 3.0])
    with pytest.raises(oracle_lib.NotSPD):
        oracle_lib.dense_chol(a)


@pytest.mark.parametrize("n,m", [(5, 1), (17, 9), (64, 40)])
def test_lower_solve_matches_numpy(oracle_lib, n, m):
    rng = np.random.default_rng(n + m)
    g = np.linalg.cholesky(_spd(rng, n, 1e3))
    b = rng.standard_normal((n, m))
    x = oracle_lib.dense_lower_solve(g, b)
    np.testing.assert_allclose(x, np.linalg.solve(g, b), rtol=1e-11, atol=1e-12)


def _reconstruct(V, tau, r):
    s = V.shape[0]
    Q = np.eye(s)
    for k in reversed(range(r)):
        v = V[:, k]
        Q = Q - tau[k] * np.outer(v, v @ Q)
    return Q


@pytest.mark.parametrize("s,w,rank,eps", [(8, 12, 3, 1e-6), (16, 40, 16, 0.0),
                                          (30, 10, 5, 1e-3), (20, 60, 4, 1e-2)])
def test_cpqr_invariants(oracle_lib, s, w, rank, eps):
    rng = np.random.default_rng(s * w)
    B = rng.standard_normal((s, rank)) @ rng.standard_normal((rank, w))
    B += 1e-5 * rng.standard_normal((s, w))
    r, V, tau, piv, RM = oracle_lib.dense_cpqr(B, eps)
    Q = _reconstruct(V, tau, r)
    # orthogonal, and RM = Q^T B (every reflector applied to every column)
    np.testing.assert_allclose(Q.T @ Q, np.eye(s), atol=1e-13)
    np.testing.assert_allclose(Q.T @ B, RM, atol=1e-12 * np.abs(B).max())
    # pivoted columns are upper triangular with non-increasing |R_kk|
    for j in range(r):
        assert np.all(np.abs(RM[j + 1:, piv[j]]) <= 1e-14 * np.abs(B).max())
    d = np.abs(RM[np.arange(r), piv])
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))
    # rank rule: smallest k with ||R[k:,k:]||_F <= eps
    rest = np.setdiff1d(np.arange(w), piv[:r])
    assert np.linalg.norm(RM[r:][:, rest]) <= eps
    if r > 0:
        prev = np.setdiff1d(np.arange(w), piv[: r - 1])
        assert np.linalg.norm(RM[r - 1:][:, prev]) > eps
    # pivot = largest trailing column norm at every step (brute force)
    Bk = B.copy()
    for k in range(r):
        cand = np.setdiff1d(np.arange(w), piv[:k])
        nrm = (Bk[k:][:, cand] ** 2).sum(0)
        best = cand[np.flatnonzero(nrm >= (1 - 1e-6) * nrm.max())[0]]
        assert piv[k] == best
        v = V[:, k]
        Bk = Bk - tau[k] * np.outer(v, v @ Bk)


def test_cpqr_matches_lapack_pivots(oracle_lib):
    """Generic matrix (no ties): pivot order and |R_kk| agree with LAPACK's
    column-pivoted QR (dgeqp3), the textbook Businger-Golub ordering."""
    rng = np.random.default_rng(11)
    B = rng.standard_normal((12, 30)) * np.logspace(0, -6, 30)
    r, V, tau, piv, RM = oracle_lib.dense_cpqr(B, 0.0)
    _, R, P = sla.qr(B, pivoting=True, mode="economic")
    assert r == 12
    assert np.array_equal(piv[:12], P[:12])
    np.testing.assert_allclose(np.abs(RM[np.arange(12), piv]), np.abs(np.diag(R)), rtol=1e-10)


def test_cpqr_zero_and_empty(oracle_lib):
    r, *_ = oracle_lib.dense_cpqr(np.zeros((5, 7)), 0.0)
    assert r == 0
    r, *_ = oracle_lib.dense_cpqr(np.ones((4, 3)), 1e9)
    assert r == 0
    B = np.ones((4, 3))
    r, *_ = oracle_lib.dense_cpqr(B, 1e-12)
    assert r == 1  # rank-1 matrix: trailing block at rounding level after one step

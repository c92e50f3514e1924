"""Pins of the whole oracle (Algorithms 1-2, PCG, GMRES) against closed forms."""
import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs


def _factor(oracle_lib, p, depth, eps, leaf=4):
    perm, lp = oracle_lib.partition(p, leaf)
    return oracle_lib.Factor(p, perm, lp, depth, eps), perm, lp


CASES = [
    ("dirichlet", lambda: inputs.grid_operator(8, 8, 4, ratio=1e4)),
    ("ice", lambda: inputs.grid_operator(8, 8, 4, ratio=1e6, sigma=1.0, seed=2, bc="ice", shelf=0.5)),
    ("vector", lambda: inputs.vector_operator(4, 4, 3, ratio=1e3, bc="ice", shelf=0.5)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("depth", [0, 1, 2])
def test_exact_at_zero_tolerance(oracle_lib, name, make, depth):
    """eps = 0: no truncation, so M^-1 = A^-1 (Algorithm 1 with exact W_i)."""
    p = make()
    f, perm, lp = _factor(oracle_lib, p, depth, 0.0)
    A = p.dense()
    xe = np.linalg.solve(A, p.b)
    z = f.apply(p.b)
    tol = max(1e-12, 100 * np.linalg.cond(A) * np.finfo(float).eps)  # rounding bound
    assert np.linalg.norm(z - xe) <= tol * np.linalg.norm(xe)
    x, it, rr, rc = f.pcg(rtol=1e-10)
    assert rc == 0 and it == 1


def test_preconditioner_symmetric_positive_definite(oracle_lib):
    """Algorithm 2 applies W^T diag(I, M_c^-1) W: symmetric, SPD when every
    Cholesky exists.  Dense check on a small ill-conditioned grid."""
    p = inputs.grid_operator(8, 8, 4, ratio=1e6, sigma=1.0, seed=4, bc="ice", shelf=0.5)
    f, _, _ = _factor(oracle_lib, p, 2, 1e-1)
    Minv = np.stack([f.apply(e) for e in np.eye(p.n)], axis=1)
    assert np.abs(Minv - Minv.T).max() <= 1e-12 * np.abs(Minv).max()
    ev = np.linalg.eigvalsh(0.5 * (Minv + Minv.T))
    assert ev[0] > 0
    # and it is not the exact inverse at this tolerance
    assert np.abs(Minv @ p.dense() - np.eye(p.n)).max() > 1e-6


def test_first_phase_is_exact_block_cholesky(oracle_lib):
    """Level 0, phase 0 clusters have no fill (A_sw = 0, Sec. 3.1): they are
    eliminated exactly.  With eps huge every later cluster keeps rank 0 and
    drops its fill, so M = A - [[0, 0], [0, S - blockdiag(S)]] with S the exact
    Schur complement of the phase-0 DOFs."""
    p = inputs.grid_operator(8, 8, 4, ratio=1e3, sigma=1.0, seed=5, bc="ice", shelf=0.5)
    f, perm, lp = _factor(oracle_lib, p, 1, 1e30)
    s0, fin, ph = f.level_info(0)
    nc = len(s0)
    assert np.all(fin == 0)
    cl = np.empty(p.n, int)
    for c in range(nc):
        cl[perm[lp[c]:lp[c + 1]]] = c
    A = p.dense()
    red = np.flatnonzero(ph[cl] == 0)
    blk = np.flatnonzero(ph[cl] != 0)
    # checkerboard: no two later clusters are adjacent in A
    sub = A[np.ix_(blk, blk)]
    same = cl[blk][:, None] == cl[blk][None, :]
    assert np.all(sub[~same] == 0)
    S = A[np.ix_(blk, blk)] - A[np.ix_(blk, red)] @ np.linalg.solve(A[np.ix_(red, red)], A[np.ix_(red, blk)])
    M = A.copy()
    M[np.ix_(blk, blk)] -= np.where(same, 0.0, S)
    z = f.apply(p.b)
    ze = np.linalg.solve(M, p.b)
    assert np.linalg.norm(z - ze) <= 1e-11 * np.linalg.norm(ze)


def test_pcg_and_gmres_converge(oracle_lib):
    p = inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    f, _, _ = _factor(oracle_lib, p, 4, 1e-2)
    x, it, rr, rc = f.pcg(rtol=1e-8)
    true = np.linalg.norm(p.b - p.matvec(x)) / np.linalg.norm(p.b)
    assert rc == 0 and true <= 1e-8 and it < 30
    xg, itg, rrg, rcg = f.gmres(rtol=1e-8, restart=50)
    trueg = np.linalg.norm(p.b - p.matvec(xg)) / np.linalg.norm(p.b)
    assert rcg == 0 and trueg <= 1e-8 and itg < 30
    assert np.linalg.norm(x - xg) <= 1e-6 * np.linalg.norm(x)


def test_smaller_tolerance_fewer_iterations(oracle_lib):
    """Sec. 5: decreasing eps increases setup cost and reduces iterations."""
    p = inputs.grid_operator(32, 32, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=1.0)
    its = []
    for eps in (1e-1, 1e-2, 1e-4):
        f, _, _ = _factor(oracle_lib, p, 6, eps)
        its.append(f.pcg(rtol=1e-8)[1])
    assert its[0] >= its[1] >= its[2] and its[0] > its[2]


def test_not_spd_reports_level_and_cluster(oracle_lib):
    """A non-SPD diagonal block stops the factorization with its location."""
    p = inputs.grid_operator(8, 8, 4, ratio=1e2)
    perm, lp = oracle_lib.partition(p, 4)
    i0 = perm[0]  # first DOF of cluster 0, which is always in the first phase
    k = np.flatnonzero((np.repeat(np.arange(p.n), np.diff(p.rowptr)) == i0) & (p.col == i0))[0]
    p.val = p.val.copy()
    p.val[k] = -1.0
    with pytest.raises(oracle_lib.NotSPD) as e:
        oracle_lib.Factor(p, perm, lp, 2, 1e-2)
    assert e.value.level == 0 and e.value.cluster == 0


def test_dirichlet_small_workload(oracle_lib):
    p = inputs.anisotropic_16x16x8()
    f, _, lp = _factor(oracle_lib, p, 4, 1e-2)
    assert len(lp) - 1 == 64
    x, it, rr, rc = f.pcg(rtol=1e-8)
    assert rc == 0 and np.linalg.norm(p.b - p.matvec(x)) <= 1e-8 * np.linalg.norm(p.b)

"""Pins of the oracle's elimination without deferred compression (plain
LoRaSp: A_sw compressed unscaled, Sec. 2 Eq. offdiag, then the fine DOFs
eliminated) and of the oracle's threaded phases.

* One step on a dense (s, n, w) matrix, followed by eliminating the coarse
  DOFs exactly, is the Schur complement of compress(A) of Eq. sc_old, formed
  from its definition (``single_step.schur_no_dc``) at the step's threshold:
  eps times the square root of the largest diagonal entry of A_ss (the
  threshold deferred compression applies when A_ss is a multiple of the
  identity, in the units of the unscaled block).
* A_sw = 0: the step is plain block Cholesky (Sec. 3.1), as with DC.
* eps = 0: nothing is dropped, M^-1 = A^-1 and PCG takes one iteration.
* eps huge: every compression keeps rank 0 in both variants, so both give the
  same preconditioner (pinned for DC by the first-phase test).
* Clusters of a phase processed on several threads give bit-identical results.
"""
import numpy as np
import pytest

from oracle import single_step as ss
from paper_1811_11248_gb300 import inputs

NS, NN, NW = 6, 5, 7


@pytest.mark.parametrize("seed", range(5))
def test_nodc_step_equals_sc_old(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    A = ss.random_spd_case(rng, NS, NN, NW, sigma_min=1e-3)
    for eps in (1e-1, 1e-2, 1e-4):
        r, K = oracle_lib.dense_step(A, NS, NN, NW, eps, nodc=True)
        St, parts = ss.schur_no_dc(A, NS, NN, eps * np.sqrt(np.diag(A)[:NS].max()))
        assert r == parts["r"]
        Acc, X, Y = K[:r, :r], K[:r, r:], K[r:, r:]
        S = Y - X.T @ np.linalg.solve(Acc, X) if r > 0 else Y
        np.testing.assert_allclose(S, St, atol=1e-9 * np.abs(A).max())
        # the coarse block is SPD and V_1^T is the coupling to w
        if r > 0:
            assert np.linalg.eigvalsh(0.5 * (Acc + Acc.T))[0] > 0
            np.testing.assert_allclose(np.abs(K[:r, r + NN:]), np.abs(parts["V1t"]), atol=1e-12 * np.abs(A).max())


def test_nodc_no_far_block_is_plain_block_cholesky(oracle_lib):
    rng = np.random.default_rng(7)
    A = ss.random_spd_case(rng, NS, NN + NW, 0)
    r, K = oracle_lib.dense_step(A, NS, NN + NW, 0, 1e-2, nodc=True)
    assert r == 0
    np.testing.assert_allclose(K, ss.schur_exact(A, NS), atol=1e-10 * np.abs(A).max())


CASES = [
    ("dirichlet", lambda: inputs.grid_operator(8, 8, 4, ratio=1e4)),
    ("ice", lambda: inputs.grid_operator(8, 8, 4, ratio=1e6, sigma=1.0, seed=2, bc="ice", shelf=0.5)),
    ("vector", lambda: inputs.vector_operator(4, 4, 3, ratio=1e3, bc="ice", shelf=0.5)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("depth", [1, 2])
def test_nodc_exact_at_zero_tolerance(oracle_lib, name, make, depth):
    p = make()
    perm, lp = oracle_lib.partition(p, 4)
    f = oracle_lib.Factor(p, perm, lp, depth, 0.0, nodc=True)
    A = p.dense()
    xe = np.linalg.solve(A, p.b)
    z = f.apply(p.b)
    tol = max(1e-12, 100 * np.linalg.cond(A) * np.finfo(float).eps)
    assert np.linalg.norm(z - xe) <= tol * np.linalg.norm(xe)
    # one PCG step reaches the rounding level of the exact inverse
    x, it, rr, rc = f.pcg(rtol=max(1e-10, tol))
    assert rc == 0 and it == 1


def test_nodc_equals_dc_when_every_rank_is_zero(oracle_lib):
    p = inputs.grid_operator(8, 8, 4, ratio=1e3, sigma=1.0, seed=5, bc="ice", shelf=0.5)
    perm, lp = oracle_lib.partition(p, 4)
    fd = oracle_lib.Factor(p, perm, lp, 2, 1e30)
    fn = oracle_lib.Factor(p, perm, lp, 2, 1e30, nodc=True)
    for l in range(2):
        assert all(np.array_equal(a, b) for a, b in zip(fd.level_info(l), fn.level_info(l)))
    r = np.random.default_rng(3).uniform(-1, 1, p.n)
    zd, zn = fd.apply(r), fn.apply(r)
    assert np.linalg.norm(zd - zn) <= 1e-12 * np.linalg.norm(zd)


def test_nodc_preconditioner_symmetric(oracle_lib):
    p = inputs.grid_operator(8, 8, 4, ratio=1e2, sigma=1.0, seed=4, bc="ice", shelf=0.5)
    perm, lp = oracle_lib.partition(p, 4)
    f = oracle_lib.Factor(p, perm, lp, 2, 1e-3, nodc=True)
    assert max(f.level_info(l)[1].max() for l in range(2)) > 0  # something was compressed
    Minv = np.stack([f.apply(e) for e in np.eye(p.n)], axis=1)
    assert np.abs(Minv - Minv.T).max() <= 1e-12 * np.abs(Minv).max()


@pytest.mark.parametrize("nodc", [False, True])
def test_threads_give_identical_factor(oracle_lib, nodc):
    p = inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    perm, lp = oracle_lib.partition(p, 4)
    f1 = oracle_lib.Factor(p, perm, lp, 4, 1e-2, nodc=nodc, threads=1)
    f4 = oracle_lib.Factor(p, perm, lp, 4, 1e-2, nodc=nodc, threads=4)
    for l in range(4):
        assert all(np.array_equal(a, b) for a, b in zip(f1.level_info(l), f4.level_info(l)))
    r = np.random.default_rng(5).uniform(-1, 1, p.n)
    assert np.array_equal(f1.apply(r), f4.apply(r))
    assert f1.top_n == f4.top_n


def test_dc_iterations_flat_under_refinement_nodc_doubling(oracle_lib):
    """The trend of Tables 5 and 6 (Sec. 5) on the extruded stand-in
    (9 layers, ratio 1e6, log-normal sigma 1, Neumann top, shelf): at eps =
    1e-2, without DC the PCG iterations grow about twofold per horizontal
    refinement; with DC they stay nearly constant and far fewer."""
    its = {}
    for nx in (16, 32):
        p = inputs.grid_operator(nx, nx, 9, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
        perm, lp = oracle_lib.partition(p, 4)
        depth = oracle_lib.default_depth(len(lp) - 1)
        for nodc in (False, True):
            f = oracle_lib.Factor(p, perm, lp, depth, 1e-2, nodc=nodc, threads=4)
            x, it, rr, rc = f.pcg(rtol=1e-8)
            assert rc == 0 and np.linalg.norm(p.b - p.matvec(x)) <= 1e-8 * np.linalg.norm(p.b)
            its[nx, nodc] = it
    print("PCG iterations (nx, nodc):", its)
    for nx in (16, 32):
        assert its[nx, True] >= 2 * its[nx, False]
    assert its[32, True] >= 1.5 * its[16, True]
    assert its[32, False] <= its[16, False] + 2

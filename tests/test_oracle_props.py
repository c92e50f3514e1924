"""Props. 1-2, the Corollary and Table 1 of Sec. 2, by brute force on small
dense SPD matrices with ill-conditioned A_ss (formed from the definitions)."""
import numpy as np
import pytest

from oracle import single_step as ss

NS, NN, NW = 8, 6, 10


def _case(seed, eps=1e-2, sigma_min=1e-4):
    rng = np.random.default_rng(seed)
    A = ss.random_spd_case(rng, NS, NN, NW, sigma_min=sigma_min)
    SA = ss.schur_exact(A, NS)
    St, pt = ss.schur_no_dc(A, NS, NN, eps)
    Sh, ph = ss.schur_dc(A, NS, NN, eps)
    return A, SA, St, pt, Sh, ph


@pytest.mark.parametrize("seed", range(6))
def test_error_closed_forms(oracle_lib, seed):
    """S_A~ - S_A equals Eq. err_old and S_(SAS)^ - S_A equals Eq. err_new."""
    A, SA, St, pt, Sh, ph = _case(seed)
    scale = np.abs(A[NS:, NS:]).max()
    Et = ss.err_old_closed_form(A, NS, NN, pt)
    Eh = ss.err_new_closed_form(A, NS, NN, ph)
    np.testing.assert_allclose(St - SA, Et, atol=1e-12 * scale)
    np.testing.assert_allclose(Sh - SA, Eh, atol=1e-12 * scale)
    # the nn block is exact in both schemes
    assert np.abs((Sh - SA)[:NN, :NN]).max() <= 1e-12 * scale


@pytest.mark.parametrize("seed", range(6))
def test_prop_bounds_and_corollary(oracle_lib, seed):
    eps = 1e-2
    A, SA, St, pt, Sh, ph = _case(seed, eps)
    Ass, Ans, Asw = A[:NS, :NS], A[NS:NS + NN, :NS], A[:NS, NS + NN:]
    smin = np.linalg.eigvalsh(Ass)[0]
    n2 = lambda m: np.linalg.norm(m, 2)
    Et, Eh = St - SA, Sh - SA
    w = slice(NN, NN + NW)
    n = slice(0, NN)
    # Prop. 2 (with ||V2|| <= ||R22||_F <= eps)
    scale = np.abs(A[NS:, NS:]).max()  # Eh is formed by cancellation at this scale
    v2 = n2(ph["V2t"])
    assert v2 <= eps * (1 + 1e-12)
    assert abs(n2(Eh[w, w]) - v2 ** 2) <= 1e-12 * scale
    assert n2(Eh[n, w]) <= eps * n2(Ans) / np.sqrt(smin) * (1 + 1e-10)
    assert n2(Eh) <= (eps * n2(Ans) / np.sqrt(smin) + eps ** 2) * (1 + 1e-10)
    # Prop. 1
    tv2 = n2(pt["V2t"])
    assert n2(Et[w, w]) <= (2 * tv2 * n2(Asw) + tv2 ** 2) / smin * (1 + 1e-8)
    assert n2(Et[n, w]) <= tv2 * n2(Ans) / smin * (1 + 1e-8)
    # Corollary: E^_ww PSD and the ww block of the DC Schur complement SPD
    assert np.linalg.eigvalsh(Eh[w, w])[0] >= -1e-12 * scale
    assert np.linalg.eigvalsh(Sh[w, w])[0] > 0


def test_dc_reduces_schur_error_when_ill_conditioned(oracle_lib):
    """Table 1: with sigma_min(A_ss) << ||A_sw|| the DC error is smaller.
    Not a theorem for every matrix: count wins over 100 seeds."""
    wins, ratios = 0, []
    for seed in range(100):
        A, SA, St, pt, Sh, ph = _case(1000 + seed, eps=1e-2, sigma_min=1e-5)
        et, eh = np.linalg.norm(St - SA, 2), np.linalg.norm(Sh - SA, 2)
        wins += eh < et
        ratios.append(eh / max(et, 1e-300))
    assert wins >= 95, (wins, np.median(ratios))
    assert np.median(ratios) < 1e-1


def test_factor_step_equals_sc_new(oracle_lib):
    """The factorization's own per-cluster routine (scaling, CPQR,
    sparsification, fine elimination, write-back) followed by eliminating the
    coarse DOFs gives Eq. sc_new formed from the definitions."""
    for seed in range(5):
        rng = np.random.default_rng(seed)
        A = ss.random_spd_case(rng, NS, NN, NW, sigma_min=1e-3)
        r, K = oracle_lib.dense_step(A, NS, NN, NW, 1e-2)
        Sh, ph = ss.schur_dc(A, NS, NN, 1e-2)
        assert r == ph["r"]
        X, Y = K[:r, r:], K[r:, r:]
        np.testing.assert_allclose(np.eye(r), K[:r, :r])
        np.testing.assert_allclose(Y - X.T @ X, Sh, atol=1e-10 * np.abs(A[NS:, NS:]).max())


def test_no_far_block_is_plain_block_cholesky(oracle_lib):
    """A_sw = 0 (Sec. 3.1): the step is ordinary block Cholesky, rank 0."""
    rng = np.random.default_rng(7)
    A = ss.random_spd_case(rng, NS, NN + NW, 0)
    r, K = oracle_lib.dense_step(A, NS, NN + NW, 0, 1e-2)
    assert r == 0
    np.testing.assert_allclose(K, ss.schur_exact(A, NS), atol=1e-10 * np.abs(A).max())

"""One elimination step with and without deferred compression (Sec. 2).

Test infrastructure only.  Every matrix here is formed from its definition in
Sec. 2 with dense numpy algebra; the low-rank decomposition is the oracle's
column-pivoted QR (``oracle.dense_cpqr``) at absolute tolerance eps, applied to
A_sw (no DC, Eq. offdiag) or to G_s^-1 A_sw (DC, Eq. offdiag_new).

Index sets: the matrix is ordered (s, n, w) with sizes (ns, nn, nw).
"""
from __future__ import annotations

import numpy as np

from . import dense_cpqr


def _blocks(A, ns, nn):
    s = slice(0, ns)
    n = slice(ns, ns + nn)
    w = slice(ns + nn, A.shape[0])
    return s, n, w


def _householder_q(V, tau, r):
    """Q = H_0 H_1 ... H_{r-1} with H_k = I - tau_k v_k v_k^T."""
    s = V.shape[0]
    Q = np.eye(s)
    for k in reversed(range(r)):
        v = V[:, k]
        Q = Q - tau[k] * np.outer(v, v @ Q)
    return Q


def lowrank(B, eps):
    """B = U V^T with U orthogonal (Eq. offdiag): returns U1, U2, V1t, V2t."""
    r, V, tau, piv, RM = dense_cpqr(B, eps)
    U = _householder_q(V, tau, r)
    return U[:, :r], U[:, r:], RM[:r, :], RM[r:, :], r


def schur_exact(A, ns):
    """S_A, the lower 2x2 block of C_s A C_s^T (Eq. exact_sc)."""
    Ass = A[:ns, :ns]
    Ars = A[ns:, :ns]
    return A[ns:, ns:] - Ars @ np.linalg.solve(Ass, Ars.T)


def schur_no_dc(A, ns, nn, eps):
    """S of compress(A) without DC (Eq. sc_old) and the parts of Eq. offdiag."""
    s, n, w = _blocks(A, ns, nn)
    U1, U2, V1t, V2t, r = lowrank(A[s, w], eps)
    At = A.copy()
    At[s, w] = U1 @ V1t
    At[w, s] = (U1 @ V1t).T
    return schur_exact(At, ns), dict(U1=U1, U2=U2, V1t=V1t, V2t=V2t, r=r)


def schur_dc(A, ns, nn, eps):
    """S of compress(S_s A S_s^T) with DC (Eq. sc_new) and its parts."""
    s, n, w = _blocks(A, ns, nn)
    G = np.linalg.cholesky(A[s, s])
    Gi = np.linalg.inv(G)
    U1, U2, V1t, V2t, r = lowrank(Gi @ A[s, w], eps)
    Sc = A.copy()  # S_s A S_s^T
    Sc[s, :] = Gi @ Sc[s, :]
    Sc[:, s] = Sc[:, s] @ Gi.T
    Sc[s, w] = U1 @ V1t
    Sc[w, s] = (U1 @ V1t).T
    return schur_exact(Sc, ns), dict(G=G, U1=U1, U2=U2, V1t=V1t, V2t=V2t, r=r)


def err_old_closed_form(A, ns, nn, parts):
    """E~ of Eq. err_old, written blockwise from its statement."""
    s, n, w = _blocks(A, ns, nn)
    U1, U2, V1t, V2t = parts["U1"], parts["U2"], parts["V1t"], parts["V2t"]
    Ass_inv = np.linalg.inv(A[s, s])
    m = A.shape[0] - ns
    E = np.zeros((m, m))
    nl = slice(0, nn)
    wl = slice(nn, m)
    E[nl, wl] = A[n, s] @ Ass_inv @ (U2 @ V2t)
    E[wl, nl] = (V2t.T @ U2.T) @ Ass_inv @ A[s, n]
    E[wl, wl] = (A[w, s] @ Ass_inv @ A[s, w]
                 - (V1t.T @ U1.T) @ Ass_inv @ (U1 @ V1t))
    return E


def err_new_closed_form(A, ns, nn, parts):
    """E^ of Eq. err_new, written blockwise from its statement."""
    s, n, w = _blocks(A, ns, nn)
    G, U2, V2t = parts["G"], parts["U2"], parts["V2t"]
    GiT = np.linalg.inv(G).T
    m = A.shape[0] - ns
    E = np.zeros((m, m))
    nl = slice(0, nn)
    wl = slice(nn, m)
    E[nl, wl] = A[n, s] @ GiT @ U2 @ V2t
    E[wl, nl] = E[nl, wl].T
    E[wl, wl] = V2t.T @ V2t
    return E


def random_spd_case(rng, ns, nn, nw, sigma_min=1e-4, far_rank=None,
                    far_noise=1e-3):
    """Random SPD matrix ordered (s, n, w) with an ill-conditioned A_ss.

    A_ss = Q diag(d) Q^T with d spanning [sigma_min, 1]; A_sn dense; A_sw
    numerically low rank (rank far_rank plus far_noise); the lower-right block
    is [A_sn A_sw]^T A_ss^-1 [A_sn A_sw] + Y Y^T + 0.1 I, so A is SPD and its
    exact Schur complement is Y Y^T + 0.1 I by construction.
    """
    Q, _ = np.linalg.qr(rng.standard_normal((ns, ns)))
    d = np.logspace(np.log10(sigma_min), 0.0, ns)
    Ass = (Q * d) @ Q.T
    Asn = rng.standard_normal((ns, nn)) / np.sqrt(ns)
    k = far_rank if far_rank is not None else max(1, ns // 3)
    Asw = (rng.standard_normal((ns, k)) @ rng.standard_normal((k, nw))
           / np.sqrt(k) + far_noise * rng.standard_normal((ns, nw)))
    Asw /= np.sqrt(nw)
    Ars = np.hstack([Asn, Asw])
    m = nn + nw
    Y = rng.standard_normal((m, m)) / np.sqrt(m)
    R = Ars.T @ np.linalg.solve(Ass, Ars) + Y @ Y.T + 0.1 * np.eye(m)
    A = np.block([[Ass, Ars], [Ars.T, R]])
    return 0.5 * (A + A.T)

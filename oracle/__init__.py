"""CPU oracle of the hierarchical solver (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path.

* ``hs_oracle.c`` (plain C, FP64, no BLAS): partition (Sec. 4.2), the phase
  rule, Algorithm 1 (factor), Algorithm 2 (apply), PCG and GMRES (Sec. 5).
* ``single_step.py`` (numpy): one elimination step with and without deferred
  compression, formed from the definitions of Sec. 2, for Props. 1-2.
* ``mlp.py`` (numpy): the rank predictor's forward/backward and Adam.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhsoracle.so")
_lib = None

OK, ERR_ARG, ERR_NOT_SPD, ERR_NOCONV, ERR_OOM = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build (gcc, -O2, IEEE FP64)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                           "-fno-fast-math", "-ffp-contract=off",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


P = ctypes.c_void_p
I32, I64, F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.or_partition_extruded.argtypes = [I64, P, P, P, P, I32, F64, P, P, P]
        L.or_factor_create.argtypes = [I64, P, P, P, I32, P, P, I32, F64, P, P, P]
        L.or_factor_create_ex.argtypes = [I64, P, P, P, I32, P, P, I32, F64, I32, I32, P, P, P]
        L.or_factor_free.argtypes = [P]
        L.or_apply.argtypes = [P, P, P]
        L.or_pcg.argtypes = [I64, P, P, P, P, P, P, F64, I32, P, P]
        L.or_gmres.argtypes = [I64, P, P, P, P, P, P, F64, I32, I32, P, P]
        for name in ("or_depth", "or_top_n"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = I32
        L.or_factor_bytes.argtypes = [P]
        L.or_factor_bytes.restype = I64
        for name in ("or_level_nc", "or_level_nphases", "or_level_nsteps"):
            getattr(L, name).argtypes = [P, I32]
            getattr(L, name).restype = I32
        L.or_level_info.argtypes = [P, I32, P, P, P]
        L.or_level_steps.argtypes = [P, I32, P, P]
        L.or_dense_chol.argtypes = [I32, P]
        L.or_dense_lower_solve.argtypes = [I32, P, I32, P]
        L.or_dense_cpqr.argtypes = [I32, I32, P, F64, P, P, P]
        L.or_dense_cpqr.restype = I32
        L.or_dense_step.argtypes = [I32, I32, I32, P, F64, P]
        L.or_dense_step.restype = I32
        L.or_dense_step_nodc.argtypes = [I32, I32, I32, P, F64, P]
        L.or_dense_step_nodc.restype = I32
        L.or_plan_level.argtypes = [I32, P, P, P, P, P, P, P, I64, P, P, I64]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(prob):
    return (np.ascontiguousarray(prob.rowptr, dtype=np.int64),
            np.ascontiguousarray(prob.col, dtype=np.int32),
            np.ascontiguousarray(prob.val, dtype=np.float64))


def partition(prob, leaf_lines=4, theta=0.5, use_coords=True):
    """Column-preserving partition -> (perm, leaf_ptr)."""
    rp, ci, va = _csr(prob)
    perm = np.zeros(prob.n, dtype=np.int32)
    leaf_ptr = np.zeros(prob.n + 1, dtype=np.int32)
    nleaf = np.zeros(1, dtype=np.int32)
    co = np.ascontiguousarray(prob.coords, dtype=np.float64) if use_coords else None
    rc = lib().or_partition_extruded(prob.n, _p(rp), _p(ci), _p(va),
                                     _p(co) if co is not None else None,
                                     int(leaf_lines), float(theta), _p(perm),
                                     _p(leaf_ptr), _p(nleaf))
    if rc != OK:
        raise RuntimeError(f"oracle partition failed: {rc}")
    return perm, leaf_ptr[: nleaf[0] + 1].copy()


def plan_level(adj_ptr, adj, size0):
    """Symbolic level plan -> (phase, vanished, end_ptr, end_adj, all_ptr, all_adj)."""
    size0 = np.ascontiguousarray(size0, dtype=np.int32)
    nc = len(size0)
    adj_ptr = np.ascontiguousarray(adj_ptr, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    aj = _p(adj) if len(adj) else None
    phase = np.empty(nc, np.int32)
    vanished = np.empty(nc, np.int32)
    end_ptr = np.empty(nc + 1, np.int64)
    all_ptr = np.empty(nc + 1, np.int64)
    lib().or_plan_level(nc, _p(adj_ptr), aj, _p(size0), _p(phase), _p(vanished), _p(end_ptr), None, 0,
                        _p(all_ptr), None, 0)
    end_adj = np.empty(max(int(end_ptr[-1]), 1), np.int32)
    all_adj = np.empty(max(int(all_ptr[-1]), 1), np.int32)
    rc = lib().or_plan_level(nc, _p(adj_ptr), aj, _p(size0), _p(phase), _p(vanished), _p(end_ptr),
                             _p(end_adj), len(end_adj), _p(all_ptr), _p(all_adj), len(all_adj))
    if rc != OK:
        raise RuntimeError(f"oracle plan failed: {rc}")
    return phase, vanished, end_ptr, end_adj[:int(end_ptr[-1])], all_ptr, all_adj[:int(all_ptr[-1])]


def default_depth(nleaf: int) -> int:
    """Elimination levels so that the last level has 8 clusters (at least 1)."""
    L = int(nleaf).bit_length() - 1
    return max(1, L - 2) if nleaf >= 2 else 0


class NotSPD(RuntimeError):
    def __init__(self, level, cluster):
        super().__init__(f"not SPD at level {level}, cluster {cluster}")
        self.level, self.cluster = level, cluster


class Factor:
    """Hierarchical_Factor (Algorithm 1) of a CSR matrix, plain FP64 on CPU."""

    def __init__(self, prob, perm, leaf_ptr, depth, tol, nodc=False, threads=1):
        """nodc: eliminate without deferred compression (plain LoRaSp: A_sw
        compressed unscaled, Sec. 2 Eq. offdiag); threads: clusters of a phase
        in parallel (the result does not depend on it)."""
        self.prob = prob
        self._rp, self._ci, self._va = _csr(prob)
        self.perm = np.ascontiguousarray(perm, dtype=np.int32)
        self.leaf_ptr = np.ascontiguousarray(leaf_ptr, dtype=np.int32)
        self.depth = int(depth)
        self.tol = float(tol)
        h = ctypes.c_void_p()
        fl, fc = np.zeros(1, np.int32), np.zeros(1, np.int32)
        rc = lib().or_factor_create_ex(prob.n, _p(self._rp), _p(self._ci),
                                       _p(self._va), len(self.leaf_ptr) - 1,
                                       _p(self.perm), _p(self.leaf_ptr),
                                       self.depth, self.tol, int(bool(nodc)), int(threads),
                                       ctypes.byref(h), _p(fl), _p(fc))
        if rc == ERR_NOT_SPD:
            raise NotSPD(int(fl[0]), int(fc[0]))
        if rc != OK:
            raise RuntimeError(f"oracle factor failed: {rc}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().or_factor_free(h)
            self._h = None

    def apply(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        lib().or_apply(self._h, _p(r), _p(z))
        return z

    def pcg(self, b=None, rtol=1e-8, maxit=1000):
        b = np.ascontiguousarray(self.prob.b if b is None else b, dtype=np.float64)
        x = np.zeros_like(b)
        it, rr = np.zeros(1, np.int32), np.zeros(1)
        rc = lib().or_pcg(self.prob.n, _p(self._rp), _p(self._ci), _p(self._va),
                          self._h, _p(b), _p(x), float(rtol), int(maxit),
                          _p(it), _p(rr))
        return x, int(it[0]), float(rr[0]), rc

    def gmres(self, b=None, rtol=1e-8, restart=50, maxit=1000):
        b = np.ascontiguousarray(self.prob.b if b is None else b, dtype=np.float64)
        x = np.zeros_like(b)
        it, rr = np.zeros(1, np.int32), np.zeros(1)
        rc = lib().or_gmres(self.prob.n, _p(self._rp), _p(self._ci), _p(self._va),
                            self._h, _p(b), _p(x), float(rtol), int(restart),
                            int(maxit), _p(it), _p(rr))
        return x, int(it[0]), float(rr[0]), rc

    @property
    def top_n(self):
        return int(lib().or_top_n(self._h))

    @property
    def factor_bytes(self):
        return int(lib().or_factor_bytes(self._h))

    def level_info(self, l):
        """Per cluster of level l: (start size, final size, phase)."""
        nc = lib().or_level_nc(self._h, l)
        s0, fi, ph = (np.zeros(nc, np.int32) for _ in range(3))
        lib().or_level_info(self._h, l, _p(s0), _p(fi), _p(ph))
        return s0, fi, ph

    def level_steps(self, l):
        """Processing order of level l and the rank of each step."""
        ns = lib().or_level_nsteps(self._h, l)
        c, r = np.zeros(ns, np.int32), np.zeros(ns, np.int32)
        lib().or_level_steps(self._h, l, _p(c), _p(r))
        return c, r

    def nphases(self, l):
        return int(lib().or_level_nphases(self._h, l))


def dense_chol(a):
    g = np.ascontiguousarray(a, dtype=np.float64).copy()
    rc = lib().or_dense_chol(g.shape[0], _p(g))
    if rc != OK:
        raise NotSPD(-1, -1)
    return g


def dense_lower_solve(g, b):
    g = np.ascontiguousarray(g, dtype=np.float64)
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    if x.ndim == 1:
        x = x[:, None].copy()
    lib().or_dense_lower_solve(g.shape[0], _p(g), x.shape[1], _p(x))
    return x


def dense_cpqr(B, eps):
    """CPQR of B at absolute tolerance eps -> (rank, V, tau, piv, RM).

    RM is B after the reflectors (rows < rank hold R in original column order).
    """
    s, w = B.shape
    M = np.ascontiguousarray(B, dtype=np.float64).copy()
    V = np.zeros((s, s))
    tau = np.zeros(s + 1)
    piv = np.zeros(s + 1, np.int32)
    r = lib().or_dense_cpqr(s, w, _p(M), float(eps), _p(V), _p(tau), _p(piv))
    return int(r), V, tau[:r].copy(), piv[:r].copy(), M


def dense_step(A, s, nn, nw, eps, nodc=False):
    """One scaled low-rank elimination on a dense (s, n, w) matrix (nodc: the
    step without deferred compression).

    Returns (rank, K) with K the matrix on (coarse DOFs, n, w) after the step.
    """
    N = s + nn + nw
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros(N * N)
    fn = lib().or_dense_step_nodc if nodc else lib().or_dense_step
    r = fn(s, nn, nw, _p(A), float(eps), _p(out))
    if r < 0:
        raise NotSPD(-1, -1)
    d = r + nn + nw
    return int(r), out[: d * d].reshape(d, d).copy()

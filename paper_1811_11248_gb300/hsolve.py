"""Thin ctypes binding of the C-ABI in include/hsolve.h (argument marshalling only).

Every step of the solver runs in the compiled library
(paper_1811_11248_gb300/_build/libhsolve.so: sm_103a kernels + host planner).
There is no fallback: if the library is missing or fails to load, ``lib()``
raises.  Pointers: numpy arrays are passed as host pointers, torch tensors as
their ``data_ptr()`` (host or device, as the call expects).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhsolve.so")

HS_OK, HS_ERR_ARG, HS_ERR_NOT_SPD, HS_ERR_NOCONV = 0, 1, 2, 3
HS_ERR_CUDA, HS_ERR_OOM, HS_ERR_UNSUPPORTED, HS_ERR_TIMEOUT = 4, 5, 6, 7
HS_MEM_HOST, HS_MEM_DEVICE = 0, 1
HS_PREC_FP64, HS_PREC_MIXED = 0, 1
HS_KRYLOV_PCG, HS_KRYLOV_GMRES = 0, 1
HS_PRODUCTS_FP32, HS_PRODUCTS_TF32X3, HS_PRODUCTS_TF32, HS_PRODUCTS_BF16 = 0, 1, 2, 3
HS_PART_AUTO, HS_PART_MULTILEVEL = 0, 1
KERNEL_CLASSES = ("factor", "schur", "assembly", "top", "apply", "krylov", "factor_fused", "spmv")

P = ctypes.c_void_p
I32, I64, F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class hs_tree(ctypes.Structure):
    _fields_ = [("n_leaf", I32), ("perm", ctypes.POINTER(I32)),
                ("leaf_ptr", ctypes.POINTER(I32)), ("depth", I32)]


class hs_options(ctypes.Structure):
    _fields_ = [("tol", F64), ("depth", I32), ("leaf_lines", I32), ("theta", F64),
                ("precision", I32), ("krylov", I32), ("restart", I32), ("rtol", F64),
                ("maxit", I32), ("mem", I32), ("profile", I32), ("stream", P), ("coords", P),
                ("coarse_dense", I32), ("fused_levels", I32), ("record_ranks", I32),
                ("rank_model", P), ("no_dc", I32), ("wait_polls", I32), ("schur_products", I32),
                ("partitioner", I32)]


class hs_info(ctypes.Structure):
    _fields_ = [("iters", I32), ("rel_resid", F64), ("setup_s", F64), ("solve_s", F64),
                ("fail_level", I32), ("fail_cluster", I32), ("factor_bytes", I64)]


class HsError(RuntimeError):
    def __init__(self, code, where, info=None):
        self.code = code
        self.info = info
        msg = lib().hs_status_str(code).decode()
        if info is not None and code == HS_ERR_NOT_SPD:
            msg += f" (level {info.fail_level}, cluster {info.fail_cluster})"
        super().__init__(f"{where}: {msg} [{code}]")


_lib = None


def lib():
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"hsolve library not built ({LIB_PATH} missing); run "
                           "python -c 'import __graft_entry__ as g; g.build()'")
    L = ctypes.CDLL(LIB_PATH)
    L.hs_default_options.argtypes = [ctypes.POINTER(hs_options)]
    L.hs_partition_extruded.argtypes = [I64, P, P, P, P, I32, F64, ctypes.POINTER(hs_tree)]
    L.hs_partition_multilevel.argtypes = [I64, P, P, P, I32, F64, ctypes.POINTER(hs_tree)]
    L.hs_tree_free.argtypes = [ctypes.POINTER(hs_tree)]
    L.hs_plan_level.argtypes = [I32, P, P, P, I32, P, P, P, P, P, I64, P, P, I64]
    L.hs_setup.argtypes = [I64, P, P, P, ctypes.POINTER(hs_tree), ctypes.POINTER(hs_options),
                           ctypes.POINTER(P), ctypes.POINTER(hs_info)]
    L.hs_apply.argtypes = [P, P, P]
    L.hs_krylov.argtypes = [P, P, P, ctypes.POINTER(hs_info)]
    L.hs_krylov_noalloc.argtypes = [P, P, P, ctypes.POINTER(hs_info)]
    L.hs_solve.argtypes = [I64, P, P, P, P, P, ctypes.POINTER(hs_options), ctypes.POINTER(hs_info)]
    L.hs_destroy.argtypes = [P]
    L.hs_num_levels.argtypes = [P, ctypes.POINTER(I32)]
    L.hs_level_clusters.argtypes = [P, I32, ctypes.POINTER(I32)]
    L.hs_level_info.argtypes = [P, I32, P, P, P]
    L.hs_top_size.argtypes = [P, ctypes.POINTER(I32)]
    L.hs_kernel_stats.argtypes = [P, I32, P, P, P, P, P]
    L.hs_reset_kernel_stats.argtypes = [P]
    L.hs_measure_fp64_peak.argtypes = [P, ctypes.POINTER(F64)]
    L.hs_measure_fp32_peak.argtypes = [P, ctypes.POINTER(F64)]
    L.hs_eval_pivot_reciprocals.argtypes = [I64, P, P, P, P]
    L.hs_launch_count.argtypes = [ctypes.POINTER(I64)]
    L.hs_setup_batched.argtypes = [I32, P, I64, P, P, P, ctypes.POINTER(hs_options), ctypes.POINTER(P),
                                   ctypes.POINTER(hs_info)]
    L.hs_krylov_batched.argtypes = [P, P, P, P, P, ctypes.POINTER(hs_info)]
    L.hs_num_problems.argtypes = [P, ctypes.POINTER(I32)]
    L.hs_problem_info.argtypes = [P, I32, P, P, P, P]
    F32 = ctypes.c_float
    L.hs_mlp_forward.argtypes = [P, P, I64, P, P]
    L.hs_mlp_grad.argtypes = [P, P, P, P, I32, P, P, P]
    L.hs_mlp_adam.argtypes = [P, P, P, P, I32, F32, P]
    L.hs_mlp_train.argtypes = [P, P, P, I64, P, I64, I32, F32, P, P]
    L.hs_rank_samples.argtypes = [P, P, P, P, ctypes.POINTER(I64)]
    L.hs_status_str.argtypes = [ctypes.c_int]
    L.hs_status_str.restype = ctypes.c_char_p
    _lib = L
    return L


# names the C-ABI exports (tests check that every one is present)
EXPORTED = ("hs_default_options", "hs_partition_extruded", "hs_tree_free", "hs_setup", "hs_apply",
            "hs_krylov", "hs_krylov_noalloc", "hs_solve", "hs_destroy", "hs_num_levels", "hs_level_clusters",
            "hs_level_info", "hs_top_size", "hs_kernel_stats", "hs_reset_kernel_stats",
            "hs_measure_fp64_peak", "hs_launch_count", "hs_status_str", "hs_setup_batched",
            "hs_krylov_batched", "hs_num_problems", "hs_problem_info", "hs_mlp_forward", "hs_mlp_grad",
            "hs_mlp_adam", "hs_mlp_train", "hs_rank_samples", "hs_plan_level", "hs_eval_pivot_reciprocals",
            "hs_measure_fp32_peak", "hs_partition_multilevel")
MLP_NIN, MLP_NPARAM, MLP_MAX_BATCH = 8, 4801, 256


def _ptr(x):
    """Host pointer of a numpy array or data_ptr() of a torch tensor (or None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(P)
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return P(x.data_ptr())
    if isinstance(x, int):
        return P(x)
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _dvec(t, n, name):
    """Pointer of a device vector argument: a contiguous CUDA float64 tensor of
    n elements (the kernels read and write exactly n doubles there, so a wrong
    buffer is refused here instead of being accessed out of bounds)."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != "torch.float64":
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return _ptr(t)


def _check(rc, where, info=None):
    if rc != HS_OK:
        raise HsError(rc, where, info)


def hs_default_options(**kw):
    o = hs_options()
    _check(lib().hs_default_options(ctypes.byref(o)), "hs_default_options")
    for k, v in kw.items():
        if k == "stream":
            v = P(v) if v is not None else None
        elif k == "coords":
            o._coords_keep = v  # the caller's array must outlive the call
            v = _ptr(v)
        elif k == "rank_model":
            v = None if v is None else np.ascontiguousarray(v, dtype=np.float32)
            o._model_keep = v
            v = _ptr(v)
        setattr(o, k, v)
    return o


def hs_partition_extruded(n, rowptr, col, val, coords=None, leaf_lines=4, theta=0.5):
    """-> (perm int32[n], leaf_ptr int32[n_leaf+1], default depth); host arrays."""
    t = hs_tree()
    _check(lib().hs_partition_extruded(int(n), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(coords),
                                       int(leaf_lines), float(theta), ctypes.byref(t)),
           "hs_partition_extruded")
    return _take_tree(t, n)


def hs_partition_multilevel(n, rowptr, col, val, leaf_lines=4, theta=0.5):
    """Partition from the matrix alone -> (perm, leaf_ptr, default depth)."""
    t = hs_tree()
    _check(lib().hs_partition_multilevel(int(n), _ptr(rowptr), _ptr(col), _ptr(val),
                                         int(leaf_lines), float(theta), ctypes.byref(t)),
           "hs_partition_multilevel")
    return _take_tree(t, n)


def _take_tree(t, n):
    try:
        perm = np.ctypeslib.as_array(t.perm, shape=(int(n),)).copy()
        lp = np.ctypeslib.as_array(t.leaf_ptr, shape=(t.n_leaf + 1,)).copy()
        depth = int(t.depth)
    finally:
        lib().hs_tree_free(ctypes.byref(t))
    return perm, lp, depth


def hs_plan_level(adj_ptr, adj, size0, ranges=None):
    """Phase plan of one level on the host ->
    (phase, vanished, end_ptr, end_adj, all_ptr, all_adj)."""
    size0 = np.ascontiguousarray(size0, dtype=np.int32)
    nc = len(size0)
    adj_ptr = np.ascontiguousarray(adj_ptr, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    rg = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int32).reshape(-1)
    nr = 0 if rg is None else len(rg) // 2
    phase = np.empty(nc, np.int32)
    vanished = np.empty(nc, np.int32)
    end_ptr = np.empty(nc + 1, np.int64)
    all_ptr = np.empty(nc + 1, np.int64)
    _check(lib().hs_plan_level(nc, _ptr(adj_ptr), _ptr(adj), _ptr(size0), nr, _ptr(rg), _ptr(phase),
                               _ptr(vanished), _ptr(end_ptr), None, 0, _ptr(all_ptr), None, 0), "hs_plan_level")
    end_adj = np.empty(max(int(end_ptr[-1]), 1), np.int32)
    all_adj = np.empty(max(int(all_ptr[-1]), 1), np.int32)
    _check(lib().hs_plan_level(nc, _ptr(adj_ptr), _ptr(adj), _ptr(size0), nr, _ptr(rg), _ptr(phase),
                               _ptr(vanished), _ptr(end_ptr), _ptr(end_adj), len(end_adj), _ptr(all_ptr),
                               _ptr(all_adj), len(all_adj)), "hs_plan_level")
    return phase, vanished, end_ptr, end_adj[:int(end_ptr[-1])], all_ptr, all_adj[:int(all_ptr[-1])]


class Handle:
    """Factor handle returned by hs_setup (owns the device factor)."""

    def __init__(self, h, n, info):
        self._h = h
        self.n = n
        self.setup_info = info

    def close(self):
        if self._h is not None and self._h.value:
            lib().hs_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hs_apply(self, r, z):
        if r.data_ptr() == z.data_ptr():
            raise ValueError("r and z may not alias")
        _check(lib().hs_apply(self._h, _dvec(r, self.n, "r"), _dvec(z, self.n, "z")), "hs_apply")

    def hs_krylov(self, b, x, check=True):
        info = hs_info()
        rc = lib().hs_krylov(self._h, _dvec(b, self.n, "b"), _dvec(x, self.n, "x"), ctypes.byref(info))
        if check:
            _check(rc, "hs_krylov", info)
        return info, rc

    def hs_krylov_noalloc(self, b, x, check=True):
        """PCG with the library's fixed device scratch (allocates nothing)."""
        info = hs_info()
        rc = lib().hs_krylov_noalloc(self._h, _dvec(b, self.n, "b"), _dvec(x, self.n, "x"), ctypes.byref(info))
        if check:
            _check(rc, "hs_krylov_noalloc", info)
        return info, rc

    def num_levels(self):
        v = I32()
        _check(lib().hs_num_levels(self._h, ctypes.byref(v)), "hs_num_levels")
        return int(v.value)

    def level_info(self, level):
        nc = I32()
        _check(lib().hs_level_clusters(self._h, int(level), ctypes.byref(nc)), "hs_level_clusters")
        s0, fi, ph = (np.zeros(nc.value, np.int32) for _ in range(3))
        _check(lib().hs_level_info(self._h, int(level), _ptr(s0), _ptr(fi), _ptr(ph)), "hs_level_info")
        return s0, fi, ph

    def top_size(self):
        v = I32()
        _check(lib().hs_top_size(self._h, ctypes.byref(v)), "hs_top_size")
        return int(v.value)

    def kernel_stats(self):
        k = len(KERNEL_CLASSES)
        t = np.zeros(k)
        n = np.zeros(k, np.int64)
        f = np.zeros(k)
        f32 = np.zeros(k)
        b = np.zeros(k)
        _check(lib().hs_kernel_stats(self._h, k, _ptr(t), _ptr(n), _ptr(f), _ptr(f32), _ptr(b)), "hs_kernel_stats")
        return {name: dict(ms=float(t[i]), launches=int(n[i]), flops=float(f[i]), flops32=float(f32[i]),
                           bytes=float(b[i]))
                for i, name in enumerate(KERNEL_CLASSES)}

    def hs_krylov_batched(self, b, x, check=True):
        """-> (info, rc, iters int32[nprob], rel_resid float64[nprob])."""
        npb = self.num_problems()
        it = np.zeros(npb, np.int32)
        rr = np.zeros(npb)
        info = hs_info()
        rc = lib().hs_krylov_batched(self._h, _dvec(b, self.n, "b"), _dvec(x, self.n, "x"), _ptr(it), _ptr(rr),
                                     ctypes.byref(info))
        if check:
            _check(rc, "hs_krylov_batched", info)
        return info, rc, it, rr

    def num_problems(self):
        v = I32()
        _check(lib().hs_num_problems(self._h, ctypes.byref(v)), "hs_num_problems")
        return int(v.value)

    def problem_info(self, prob):
        """-> (leaf_lo, leaf_hi, depth, ntop) of problem prob."""
        v = [I32() for _ in range(4)]
        _check(lib().hs_problem_info(self._h, int(prob), *[ctypes.byref(x) for x in v]), "hs_problem_info")
        return tuple(int(x.value) for x in v)

    def rank_samples(self):
        """-> (features float32[k, 8], rank int32[k], size int32[k])."""
        cnt = I64()
        _check(lib().hs_rank_samples(self._h, None, None, None, ctypes.byref(cnt)), "hs_rank_samples")
        k = int(cnt.value)
        f = np.zeros((k, 8), np.float32)
        r = np.zeros(k, np.int32)
        s = np.zeros(k, np.int32)
        _check(lib().hs_rank_samples(self._h, _ptr(f), _ptr(r), _ptr(s), ctypes.byref(cnt)), "hs_rank_samples")
        return f, r, s

    def reset_kernel_stats(self):
        _check(lib().hs_reset_kernel_stats(self._h), "hs_reset_kernel_stats")


def hs_setup(n, rowptr, col, val, tree=None, opt=None, **kw):
    """tree: None or (perm, leaf_ptr, depth) host arrays."""
    opt = opt if opt is not None else hs_default_options(**kw)
    info = hs_info()
    h = P()
    tp = None
    keep = None
    if tree is not None:
        perm, lp, depth = tree
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        lp = np.ascontiguousarray(lp, dtype=np.int32)
        keep = (perm, lp)
        tp = hs_tree(len(lp) - 1, perm.ctypes.data_as(ctypes.POINTER(I32)),
                     lp.ctypes.data_as(ctypes.POINTER(I32)), int(depth))
    rc = lib().hs_setup(int(n), _ptr(rowptr), _ptr(col), _ptr(val),
                        ctypes.byref(tp) if tp is not None else None, ctypes.byref(opt),
                        ctypes.byref(h), ctypes.byref(info))
    del keep
    _check(rc, "hs_setup", info)
    return Handle(h, int(n), info)


def hs_setup_batched(prob_ptr, n, rowptr, col, val, opt=None, **kw):
    """Batched setup of a block-diagonal CSR; prob_ptr: host int64[nprob + 1]."""
    opt = opt if opt is not None else hs_default_options(**kw)
    pp = np.ascontiguousarray(prob_ptr, dtype=np.int64)
    info = hs_info()
    h = P()
    rc = lib().hs_setup_batched(len(pp) - 1, _ptr(pp), int(n), _ptr(rowptr), _ptr(col), _ptr(val),
                                ctypes.byref(opt), ctypes.byref(h), ctypes.byref(info))
    _check(rc, "hs_setup_batched", info)
    return Handle(h, int(n), info)


def hs_solve(n, rowptr, col, val, b, x, opt=None, check=True, **kw):
    opt = opt if opt is not None else hs_default_options(**kw)
    info = hs_info()
    rc = lib().hs_solve(int(n), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x),
                        ctypes.byref(opt), ctypes.byref(info))
    if check:
        _check(rc, "hs_solve", info)
    return info, rc


def hs_launch_count():
    v = I64()
    _check(lib().hs_launch_count(ctypes.byref(v)), "hs_launch_count")
    return int(v.value)


def hs_eval_pivot_reciprocals(x, rsqrt_out, rcp_out, stream=None):
    """Device tensors of n float64: the factor kernels' 1/sqrt(x) and 1/x."""
    n = x.numel()
    _check(lib().hs_eval_pivot_reciprocals(n, _dvec(x, n, "x"), _dvec(rsqrt_out, n, "rsqrt_out"),
                                           _dvec(rcp_out, n, "rcp_out"), P(stream) if stream else None),
           "hs_eval_pivot_reciprocals")


def hs_measure_fp32_peak(stream=None):
    v = F64()
    _check(lib().hs_measure_fp32_peak(P(stream) if stream else None, ctypes.byref(v)),
           "hs_measure_fp32_peak")
    return float(v.value)


def hs_measure_fp64_peak(stream=None):
    v = F64()
    _check(lib().hs_measure_fp64_peak(P(stream) if stream else None, ctypes.byref(v)),
           "hs_measure_fp64_peak")
    return float(v.value)


def hs_mlp_forward(params, x, n, y, stream=None):
    """Device pointers (torch tensors): params float32[4801], x float32[n, 8] -> y float32[n]."""
    _check(lib().hs_mlp_forward(_ptr(params), _ptr(x), int(n), _ptr(y), P(stream) if stream else None),
           "hs_mlp_forward")


def hs_mlp_grad(params, x, t, idx, batch, grad, loss, stream=None):
    _check(lib().hs_mlp_grad(_ptr(params), _ptr(x), _ptr(t), _ptr(idx), int(batch), _ptr(grad), _ptr(loss),
                             P(stream) if stream else None), "hs_mlp_grad")


def hs_mlp_adam(params, grad, m, v, step, lr, stream=None):
    _check(lib().hs_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr),
                             P(stream) if stream else None), "hs_mlp_adam")


def hs_mlp_train(params, x, t, order, batch, lr, stream=None):
    """Host arrays: params float32[4801] (copied; the trained vector is
    returned), x float32[n, 8], t float32[n], order int32[nsteps * batch].
    -> (params, losses float32[nsteps])."""
    th = np.ascontiguousarray(params, dtype=np.float32).copy()
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    nsteps = len(order) // int(batch)
    losses = np.zeros(max(nsteps, 1), np.float32)
    _check(lib().hs_mlp_train(_ptr(th), _ptr(x), _ptr(t), len(t), _ptr(order), nsteps, int(batch), float(lr),
                              _ptr(losses), P(stream) if stream else None), "hs_mlp_train")
    return th, losses[:nsteps]

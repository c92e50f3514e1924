"""The allocation-free PCG entry point (hs_krylov_noalloc) against hs_krylov.

hs_krylov_noalloc serves callers that cannot allocate device memory when they
solve (a host application whose own allocator owns the device, or a loop that
must not call cudaMalloc/cudaFree after initialisation).  Its work vectors live
in a fixed array inside the library, so every call reuses memory the previous
call wrote; these tests make consecutive calls and compare each with the
allocating entry point on the same handle, within the Krylov tolerance the
other parity tests use (solution to 1e-6 relative, iterations within 1).
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1811_11248_gb300 import build, hsolve
    build.build()
    hsolve.lib()
    assert torch.cuda.is_available()
    return hsolve


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _setup(hs, p, **kw):
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, coords=np.ascontiguousarray(p.coords),
                                stream=torch.cuda.current_stream().cuda_stream, **kw)
    return hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt)


def _device_memory():
    """(bytes in use in the device's default memory pool, free device bytes),
    read through the CUDA driver API: the library allocates from that pool
    (cudaMallocAsync), and any cudaMalloc would lower the free memory."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used = ctypes.c_uint64()
    CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
    assert cu.cuMemPoolGetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_CURRENT, ctypes.byref(used)) == 0
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
    return int(used.value), int(free.value)


def _close(x, xr, info, info_r):
    assert abs(info.iters - info_r.iters) <= 1
    assert info.rel_resid <= 1e-8
    assert torch.linalg.norm(x - xr) <= 1e-6 * torch.linalg.norm(xr)


def test_noalloc_matches_krylov_on_consecutive_calls(hs):
    p = inputs.grid_operator(32, 32, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    h = _setup(hs, p)
    b1 = _dev(p.b)
    b2 = _dev(np.random.default_rng(7).uniform(-1, 1, p.n))
    ref1 = torch.empty_like(b1)
    ref2 = torch.empty_like(b1)
    info_r1, _ = h.hs_krylov(b1, ref1)
    info_r2, _ = h.hs_krylov(b2, ref2)
    cases = ((b1, ref1, info_r1), (b1, ref1, info_r1), (b2, ref2, info_r2), (b1, ref1, info_r1))
    xs = [torch.full_like(b1, float("nan")) for _ in cases]  # outputs must be fully written
    out = []
    for k, (b, _, _) in enumerate(cases):
        out.append(h.hs_krylov_noalloc(b, xs[k]))
        torch.cuda.synchronize()
        if k == 0:  # after the first call (which looks up the scratch address)
            mem = _device_memory()
    # calls 2-4 allocated nothing: the pool's usage and the free memory are unchanged
    assert _device_memory() == mem
    for (info, rc), x, (_, ref, info_r) in zip(out, xs, cases):
        assert rc == 0
        _close(x, ref, info, info_r)

    # a second handle of another size reuses the array; then the first again
    p2 = inputs.grid_operator(16, 16, 8, ratio=1e5, sigma=0.5, seed=3, bc="ice", shelf=0.5)
    h2 = _setup(hs, p2)
    c = _dev(p2.b)
    ref_c = torch.empty_like(c)
    info_rc, _ = h2.hs_krylov(c, ref_c)
    xc = torch.full_like(c, float("nan"))
    info, rc = h2.hs_krylov_noalloc(c, xc)
    torch.cuda.synchronize()
    assert rc == 0
    _close(xc, ref_c, info, info_rc)
    x = torch.full_like(b1, float("nan"))
    info, rc = h.hs_krylov_noalloc(b1, x)
    torch.cuda.synchronize()
    assert rc == 0
    _close(x, ref1, info, info_r1)
    h2.close()
    h.close()


def test_noalloc_rejects_oversized_and_gmres(hs):
    big = inputs.grid_operator(128, 128, 17, ratio=1e4)  # n = 278,528 > 262,144
    assert big.n > 262144
    h = _setup(hs, big)
    b = _dev(big.b)
    x = torch.zeros_like(b)
    info, rc = h.hs_krylov_noalloc(b, x, check=False)
    assert rc == hs.HS_ERR_ARG
    assert torch.count_nonzero(x) == 0  # rejected before any device work
    h.close()
    small = inputs.grid_operator(8, 8, 4, ratio=1e3)
    hg = _setup(hs, small, krylov=hs.HS_KRYLOV_GMRES)
    bs = _dev(small.b)
    info, rc = hg.hs_krylov_noalloc(bs, torch.zeros_like(bs), check=False)
    assert rc == hs.HS_ERR_UNSUPPORTED
    hg.close()
    # a batched handle: its problems stop one by one, which this PCG does not do
    pp, A = inputs.batched_workload(2)
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, coords=np.ascontiguousarray(A.coords),
                                stream=torch.cuda.current_stream().cuda_stream)
    hb = hs.hs_setup_batched(pp, A.n, A.rowptr, A.col, A.val, opt=opt)
    bb = _dev(A.b)
    xb = torch.zeros_like(bb)
    info, rc = hb.hs_krylov_noalloc(bb, xb, check=False)
    assert rc == hs.HS_ERR_UNSUPPORTED
    assert torch.count_nonzero(xb) == 0
    hb.close()


def test_noalloc_rejects_bad_vectors(hs):
    p = inputs.grid_operator(8, 8, 4, ratio=1e3)
    h = _setup(hs, p)
    b = _dev(p.b)
    with pytest.raises(ValueError):
        h.hs_krylov_noalloc(b[:-1], torch.zeros_like(b))  # too short
    with pytest.raises(ValueError):
        h.hs_krylov_noalloc(b, torch.zeros(p.n, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        h.hs_krylov_noalloc(b.cpu(), torch.zeros_like(b))
    h.close()

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
    for b, ref, info_r in ((b1, ref1, info_r1), (b1, ref1, info_r1), (b2, ref2, info_r2), (b1, ref1, info_r1)):
        x = torch.full_like(b, float("nan"))  # output must be fully written
        info, rc = h.hs_krylov_noalloc(b, x)
        torch.cuda.synchronize()
        assert rc == 0
        _close(x, ref, info, info_r)
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

"""Bounded device waits.  The coarse levels run all their phases in one
cooperative launch with a grid barrier between phases; every wait at that
barrier is bounded.  With options.wait_polls < 0 the first CTA that has to
wait gives up at once (a wait made to run out, no fault): the launch must
return promptly, the call must report HS_ERR_TIMEOUT without a handle, and
the GPU context must stay usable for the next setup and solve."""
import time

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


def test_barrier_timeout_returns_promptly_and_context_survives(hs):
    p = inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    st = torch.cuda.current_stream().cuda_stream
    kw = dict(tol=1e-2, mem=hs.HS_MEM_HOST, coords=np.ascontiguousarray(p.coords), stream=st)
    opt = hs.hs_default_options(wait_polls=-1, **kw)
    t0 = time.perf_counter()
    with pytest.raises(hs.HsError) as e:
        hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt)
    dt = time.perf_counter() - t0
    assert e.value.code == hs.HS_ERR_TIMEOUT
    assert dt < 2.0, dt  # returned without running out a second-long wait per phase
    torch.cuda.synchronize()
    # the next setup and solve on the same context work as usual
    h = hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=hs.hs_default_options(**kw))
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    info, rc = h.hs_krylov(torch.from_numpy(p.b).cuda(), x)
    assert rc == 0 and info.rel_resid <= 1e-8
    res = np.linalg.norm(p.b - p.matvec(x.cpu().numpy())) / np.linalg.norm(p.b)
    assert res <= 1e-8
    h.close()


def test_default_wait_limit_does_not_trigger(hs):
    """The default limit (about a second of polling) never fires in a normal
    factorization: a positive explicit limit large enough behaves the same."""
    p = inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    st = torch.cuda.current_stream().cuda_stream
    for polls in (0, 1 << 22):
        opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, coords=np.ascontiguousarray(p.coords), stream=st,
                                    wait_polls=polls)
        h = hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt)
        h.close()

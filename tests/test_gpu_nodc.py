"""GPU parity of the elimination without deferred compression (options.no_dc:
the original LoRaSp step that Sec. 2 compares against) with the oracle's
no-DC factorization, on the same seeded inputs and partition tree, and the
comparison of the two schemes that Tables 5 and 6 report.

Bars as for the deferred-compression path: identical phases and ranks per
cluster, operator parity within max(1e-10, 100 u kappa(A)) over 8 random
vectors, PCG iterations within 1, true residuals <= 1e-8, solutions within
1e-6.
"""
import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = np.finfo(float).eps


@pytest.fixture(scope="module")
def hs():
    from paper_1811_11248_gb300 import build, hsolve
    build.build()
    hsolve.lib()
    assert torch.cuda.is_available()
    return hsolve


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def setup_both(hs, oracle_lib, p, depth, tol, nodc=True, precision=0):
    perm, lp = oracle_lib.partition(p, 4)
    if depth is None:
        depth = oracle_lib.default_depth(len(lp) - 1)
    ref = oracle_lib.Factor(p, perm, lp, depth, tol, nodc=nodc, threads=4)
    opt = hs.hs_default_options(tol=tol, mem=hs.HS_MEM_DEVICE, stream=torch.cuda.current_stream().cuda_stream,
                                no_dc=int(nodc), precision=precision)
    h = hs.hs_setup(p.n, dev(p.rowptr), dev(p.col), dev(p.val), tree=(perm, lp, depth), opt=opt)
    return h, ref, depth


def check_structure(h, ref, depth):
    assert h.num_levels() == depth
    for l in range(depth):
        s0, fi, ph = h.level_info(l)
        o0, of, oph = ref.level_info(l)
        assert np.array_equal(s0, o0), f"level {l} sizes"
        assert np.array_equal(ph, oph), f"level {l} phases"
        bad = np.flatnonzero(fi != of)
        assert bad.size == 0, f"level {l} ranks differ at {bad[:10]}: {fi[bad[:10]]} vs {of[bad[:10]]}"
    assert h.top_size() == ref.top_n


def operator_diff(h, ref, n, nvec=8, seed=0):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(nvec):
        r = rng.uniform(-1, 1, n)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        h.hs_apply(dev(r), z)
        torch.cuda.synchronize()
        zo = ref.apply(r)
        worst = max(worst, np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo))
    return worst


def pcg_both(h, ref, p):
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    info, rc = h.hs_krylov(dev(p.b), x)
    xg = x.cpu().numpy()
    xo, ito, rro, rco = ref.pcg(rtol=1e-8)
    assert rco == 0
    res = np.linalg.norm(p.b - p.matvec(xg)) / np.linalg.norm(p.b)
    assert res <= 1e-8 and info.rel_resid <= 1e-8
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    return info.iters, ito


CASES = [
    ("ice-16x16x8-1e-2", lambda: inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5), 4, 1e-2),
    ("ice-16x16x8-1e-4", lambda: inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5), 4, 1e-4),
    ("ragged-12x10x5-1e-3", lambda: inputs.grid_operator(12, 10, 5, ratio=1e3, sigma=1.0, seed=2, bc="ice", shelf=0.5), 2, 1e-3),
    ("vector-8x8x4-1e-3", lambda: inputs.vector_operator(8, 8, 4, ratio=1e4, bc="ice", shelf=0.5), 2, 1e-3),
    ("exact-8x8x4", lambda: inputs.grid_operator(8, 8, 4, ratio=1e3, sigma=1.0, seed=4, bc="ice", shelf=0.5), 2, 0.0),
    ("lowratio-16x16x8-1e-3", lambda: inputs.grid_operator(16, 16, 8, ratio=1e2, sigma=1.0, seed=6, bc="ice", shelf=0.5), 4, 1e-3),
]


@pytest.mark.parametrize("name,make,depth,tol", CASES, ids=[c[0] for c in CASES])
def test_nodc_parity(hs, oracle_lib, name, make, depth, tol):
    p = make()
    h, ref, depth = setup_both(hs, oracle_lib, p, depth, tol)
    check_structure(h, ref, depth)
    bound = max(1e-10, 100 * U * np.linalg.cond(p.dense()))
    d = operator_diff(h, ref, p.n)
    assert d <= bound, (d, bound)
    itg, ito = pcg_both(h, ref, p)
    assert abs(itg - ito) <= 1, (itg, ito)
    h.close()


def test_nodc_parity_32x32x9_several_tiles(hs, oracle_lib):
    """256 leaves, 6 levels, ranks above zero on several levels."""
    p = inputs.grid_operator(32, 32, 9, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    h, ref, depth = setup_both(hs, oracle_lib, p, None, 1e-4)
    check_structure(h, ref, depth)
    assert max(ref.level_info(l)[1].max() for l in range(depth)) > 0
    d = operator_diff(h, ref, p.n, nvec=4)
    assert d <= 1e-8, d
    itg, ito = pcg_both(h, ref, p)
    assert abs(itg - ito) <= 1, (itg, ito)
    h.close()


def test_dc_against_nodc_under_refinement(hs, oracle_lib):
    """Tables 5 and 6 on the stand-in (9 layers, ratio 1e6, eps 1e-2): the
    GPU's PCG iterations equal the oracle's (within 1) in both schemes;
    without DC they grow about twofold per refinement, with DC they stay
    nearly flat and far fewer."""
    its = {}
    for nx in (16, 32, 64):
        p = inputs.grid_operator(nx, nx, 9, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
        for nodc in (False, True):
            h, ref, depth = setup_both(hs, oracle_lib, p, None, 1e-2, nodc=nodc)
            itg, ito = pcg_both(h, ref, p)
            assert abs(itg - ito) <= 1, (nx, nodc, itg, ito)
            its[nx, nodc] = itg
            h.close()
    print("GPU PCG iterations (nx, nodc):", its)
    for nx in (16, 32, 64):
        assert its[nx, True] >= 2 * its[nx, False]
    assert its[64, True] >= 3 * its[16, True]
    assert its[64, False] <= its[16, False] + 3


def test_nodc_rejects_predictor_options(hs):
    p = inputs.grid_operator(8, 8, 4, ratio=1e3)
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, no_dc=1, record_ranks=1,
                                stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(hs.HsError) as e:
        hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt)
    assert e.value.code == hs.HS_ERR_UNSUPPORTED

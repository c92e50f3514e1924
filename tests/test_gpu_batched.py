"""GPU parity of the batched path: several independent problems of uneven
size and depth in one handle (one launch sequence per level for all of
them) against the CPU oracle run on each problem alone.

Bars, per problem: identical phases and ranks per cluster, identical top
size, operator parity <= max(1e-10, 100 u kappa(A_p)), PCG iterations within
1 of the oracle's, true residual <= 1e-8 and ||x - x_or|| <= 1e-6 ||x_or||.
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


def mixed_batch():
    """Depths 1 to 5, Dirichlet and ice-sheet boundaries, ragged sizes."""
    g = inputs.grid_operator
    return [
        g(16, 16, 6, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5),
        g(8, 8, 4, ratio=1e4),
        g(12, 10, 5, ratio=1e3, sigma=1.0, seed=2, bc="ice", shelf=0.5),
        g(24, 16, 6, ratio=1e5, sigma=1.0, seed=3, bc="ice", shelf=0.5),
        g(16, 32, 5, ratio=1e6, sigma=0.5, seed=4, bc="ice", shelf=0.5),
        g(10, 12, 7, ratio=1e4, sigma=1.0, seed=5, bc="ice", shelf=0.5),
        g(4, 4, 3, ratio=1e2),
    ]


def oracle_factors(oracle_lib, probs, tol):
    refs = []
    for p in probs:
        perm, lp = oracle_lib.partition(p, 4)
        depth = oracle_lib.default_depth(len(lp) - 1)
        refs.append((oracle_lib.Factor(p, perm, lp, depth, tol), depth, len(lp) - 1))
    return refs


def setup_batched(hs, pp, A, tol, **kw):
    opt = hs.hs_default_options(tol=tol, mem=hs.HS_MEM_DEVICE, coords=A.coords,
                                stream=torch.cuda.current_stream().cuda_stream, **kw)
    return hs.hs_setup_batched(pp, A.n, dev(A.rowptr), dev(A.col), dev(A.val), opt=opt)


def check_batched_structure(h, refs):
    """Level l of the handle = level l of every problem still active, in order."""
    assert h.num_problems() == len(refs)
    D = max(d for _, d, _ in refs)
    assert h.num_levels() == D
    for l in range(D):
        s0, fi, ph = h.level_info(l)
        o = 0
        for k, (ref, depth, nleaf) in enumerate(refs):
            if depth <= l:
                continue
            m = nleaf >> l
            r0, rf, rph = ref.level_info(l)
            assert np.array_equal(s0[o:o + m], r0), f"problem {k} level {l} sizes"
            assert np.array_equal(ph[o:o + m], rph), f"problem {k} level {l} phases"
            assert np.array_equal(fi[o:o + m], rf), f"problem {k} level {l} ranks"
            o += m
        assert o == len(s0)
    lo = 0
    for k, (ref, depth, nleaf) in enumerate(refs):
        leaf_lo, leaf_hi, d, ntop = h.problem_info(k)
        assert (leaf_lo, leaf_hi, d, ntop) == (lo, lo + nleaf, depth, ref.top_n)
        lo += nleaf


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_batched_parity(hs, oracle_lib, tol):
    probs = mixed_batch()
    pp, A = inputs.block_diagonal(probs)
    refs = oracle_factors(oracle_lib, probs, tol)
    h = setup_batched(hs, pp, A, tol)
    check_batched_structure(h, refs)
    rng = np.random.default_rng(7)
    for _ in range(4):
        r = rng.uniform(-1, 1, A.n)
        z = torch.empty(A.n, dtype=torch.float64, device="cuda")
        h.hs_apply(dev(r), z)
        torch.cuda.synchronize()
        zg = z.cpu().numpy()
        for k, (p, (ref, _, _)) in enumerate(zip(probs, refs)):
            zo = ref.apply(r[pp[k]:pp[k + 1]])
            kap = np.linalg.cond(p.dense())
            d = np.linalg.norm(zg[pp[k]:pp[k + 1]] - zo) / np.linalg.norm(zo)
            assert d <= max(1e-10, 100 * U * kap), (k, d)
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info, rc, its, rel = h.hs_krylov_batched(dev(A.b), x)
    xg = x.cpu().numpy()
    for k, (p, (ref, _, _)) in enumerate(zip(probs, refs)):
        xo, ito, rro, rco = ref.pcg(rtol=1e-8)
        assert rco == 0
        assert abs(int(its[k]) - ito) <= 1, (k, its[k], ito)
        xk = xg[pp[k]:pp[k + 1]]
        assert np.linalg.norm(p.b - p.matvec(xk)) <= 1e-8 * np.linalg.norm(p.b)
        assert rel[k] <= 1e-8
        assert np.linalg.norm(xk - xo) <= 1e-6 * np.linalg.norm(xo)
    assert info.iters == its.max()
    h.close()


def test_batched_workload_problems(hs, oracle_lib):
    """The first problems of the 256-problem workload (grids 16x16x4 to
    48x48x12, ratio 1e3 to 1e6), FP64 and mixed precision."""
    probs = [inputs.batched_problem(k) for k in range(4)]
    pp, A = inputs.block_diagonal(probs)
    refs = oracle_factors(oracle_lib, probs, 1e-2)
    h = setup_batched(hs, pp, A, 1e-2)
    check_batched_structure(h, refs)
    hm = setup_batched(hs, pp, A, 1e-2, precision=hs.HS_PREC_MIXED)
    for hh, slack in ((h, 1), (hm, 3)):
        x = torch.empty(A.n, dtype=torch.float64, device="cuda")
        info, rc, its, rel = hh.hs_krylov_batched(dev(A.b), x)
        xg = x.cpu().numpy()
        for k, (p, (ref, _, _)) in enumerate(zip(probs, refs)):
            _, ito, _, _ = ref.pcg(rtol=1e-8)
            assert abs(int(its[k]) - ito) <= slack, (k, its[k], ito)
            xk = xg[pp[k]:pp[k + 1]]
            assert np.linalg.norm(p.b - p.matvec(xk)) <= 1e-8 * np.linalg.norm(p.b)
    h.close()
    hm.close()


@pytest.mark.slow
def test_batched_workload_32_problems(hs, oracle_lib):
    """32 problems spread over the 256-problem workload (every eighth), in
    one handle: per problem the phases and ranks of the oracle run on that
    problem alone, PCG iterations within 1 of the oracle's, true residuals
    <= 1e-8 and solutions within 1e-6 (FP64); the mixed form reaches 1e-8
    within 3 iterations of the oracle."""
    probs = [inputs.batched_problem(k) for k in range(0, 256, 8)]
    pp, A = inputs.block_diagonal(probs)
    refs = oracle_factors(oracle_lib, probs, 1e-2)
    h = setup_batched(hs, pp, A, 1e-2)
    check_batched_structure(h, refs)
    hm = setup_batched(hs, pp, A, 1e-2, precision=hs.HS_PREC_MIXED)
    for hh, slack in ((h, 1), (hm, 3)):
        x = torch.empty(A.n, dtype=torch.float64, device="cuda")
        info, rc, its, rel = hh.hs_krylov_batched(dev(A.b), x)
        xg = x.cpu().numpy()
        for k, (p, (ref, _, _)) in enumerate(zip(probs, refs)):
            xo, ito, _, _ = ref.pcg(rtol=1e-8)
            assert abs(int(its[k]) - ito) <= slack, (k, its[k], ito)
            xk = xg[pp[k]:pp[k + 1]]
            assert np.linalg.norm(p.b - p.matvec(xk)) <= 1e-8 * np.linalg.norm(p.b)
            if slack == 1:
                assert np.linalg.norm(xk - xo) <= 1e-6 * np.linalg.norm(xo)
    h.close()
    hm.close()


def test_batched_krylov_entry_and_zero_rhs(hs, oracle_lib):
    """hs_krylov on a batched handle runs the per-problem PCG; a problem with
    b = 0 returns x = 0 after no iteration."""
    probs = mixed_batch()[:3]
    probs[1].b = np.zeros(probs[1].n)
    pp, A = inputs.block_diagonal(probs)
    h = setup_batched(hs, pp, A, 1e-2)
    x1 = torch.empty(A.n, dtype=torch.float64, device="cuda")
    x2 = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info1, _ = h.hs_krylov(dev(A.b), x1)
    info2, _, its, rel = h.hs_krylov_batched(dev(A.b), x2)
    assert torch.equal(x1, x2)
    assert its[1] == 0 and rel[1] == 0.0
    assert torch.count_nonzero(x2[pp[1]:pp[2]]) == 0
    h.close()


def test_batched_rejects_coupled_problems(hs):
    """An entry between two problems, or a problem with a single leaf, is an
    argument error found on the host."""
    probs = mixed_batch()[:2]
    pp, A = inputs.block_diagonal(probs)
    col = A.col.copy()
    col[0] = pp[1]  # row 0 of problem 0 now points into problem 1
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST)
    with pytest.raises(hs.HsError) as e:
        hs.hs_setup_batched(pp, A.n, A.rowptr, col, A.val, opt=opt)
    assert e.value.code == hs.HS_ERR_ARG
    tiny = inputs.grid_operator(2, 2, 3, ratio=1e2)
    pp2, B = inputs.block_diagonal([probs[0], tiny])
    with pytest.raises(hs.HsError) as e:
        hs.hs_setup_batched(pp2, B.n, B.rowptr, B.col, B.val, opt=opt)
    assert e.value.code == hs.HS_ERR_ARG

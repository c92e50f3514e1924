"""GPU parity on unstructured extruded meshes (Sec. 4: the ice-sheet meshes
are unstructured triangulations extruded in layers) with the clusters taken
from the matrix alone (Sec. 4.2 with the multilevel graph bisection of
hs_partition_multilevel in place of coordinates; Sec. 6 on black-box use).

The CUDA path and the oracle factor the same tree.  Bars as in the
structured parity tests: identical phases and ranks per cluster, operator
parity within max(1e-10, 100 u kappa(A)) (kappa dense for the small cases,
1e-8 for the larger one), Krylov iterations within 1 and true residuals
<= 1e-8; the mixed form within 5 % of the ranks and 2 iterations."""
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


def stream():
    return torch.cuda.current_stream().cuda_stream


def setup_pair(hs, oracle_lib, p, tol, leaf=4, threads=1, **kw):
    perm, lp, depth = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, leaf, 0.5)
    ref = oracle_lib.Factor(p, perm, lp, depth, tol, threads=threads)
    opt = hs.hs_default_options(tol=tol, mem=hs.HS_MEM_DEVICE, stream=stream(), **kw)
    h = hs.hs_setup(p.n, dev(p.rowptr), dev(p.col), dev(p.val), tree=(perm, lp, depth), opt=opt)
    return h, ref, depth


def rank_diff(h, ref, depth, exact=True):
    assert h.num_levels() == depth
    nd = nt = 0
    for l in range(depth):
        s0, fi, ph = h.level_info(l)
        o0, of, oph = ref.level_info(l)
        assert np.array_equal(s0, o0), f"level {l} sizes"
        if exact:
            assert np.array_equal(ph, oph), f"level {l} phases"
            bad = np.flatnonzero(fi != of)
            assert bad.size == 0, f"level {l} ranks differ at {bad[:10]}: {fi[bad[:10]]} vs {of[bad[:10]]}"
        nd += int(np.sum(fi != of))
        nt += len(of)
    if exact:
        assert h.top_size() == ref.top_n
    return nd, nt


def operator_diff(h, ref, n, nvec=6, seed=0):
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


def solve(h, p):
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    info, rc = h.hs_krylov(dev(p.b), x)
    xg = x.cpu().numpy()
    res = np.linalg.norm(p.b - p.matvec(xg)) / np.linalg.norm(p.b)
    return info, rc, xg, res


SMALL = [
    ("ice-24x20x6-1e-2", lambda: inputs.unstructured_operator(24, 20, 6, ratio=1e5, sigma=1.0, seed=3), 1e-2, 4),
    ("ice-shelf-20x18x8-1e-4",
     lambda: inputs.unstructured_operator(20, 18, 8, ratio=1e6, sigma=1.0, seed=5, shelf=0.5), 1e-4, 4),
    ("dirichlet-22x21x5-1e-1",
     lambda: inputs.unstructured_operator(22, 21, 5, ratio=1e4, seed=8, bc="dirichlet"), 1e-1, 4),
    ("ragged-leaves-17x15x4", lambda: inputs.unstructured_operator(17, 15, 4, ratio=1e5, sigma=1.0, seed=2), 1e-2, 7),
    ("exact-14x12x4", lambda: inputs.unstructured_operator(14, 12, 4, ratio=1e3, sigma=1.0, seed=4), 0.0, 4),
]


@pytest.mark.parametrize("name,make,tol,leaf", SMALL, ids=[c[0] for c in SMALL])
def test_small_unstructured_parity(hs, oracle_lib, name, make, tol, leaf):
    p = make()
    h, ref, depth = setup_pair(hs, oracle_lib, p, tol, leaf=leaf)
    rank_diff(h, ref, depth)
    ev = np.linalg.eigvalsh(p.dense())
    bound = max(1e-10, 100 * U * ev[-1] / ev[0])
    d = operator_diff(h, ref, p.n)
    assert d <= bound, (d, bound)
    info, rc, xg, res = solve(h, p)
    xo, ito, rro, rco = ref.pcg(rtol=1e-8)
    assert rc == 0 and rco == 0
    assert abs(info.iters - ito) <= 1, (info.iters, ito)
    assert res <= 1e-8 and info.rel_resid <= 1e-8
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    h.close()


def test_unstructured_64x64x8_fp64_and_mixed(hs, oracle_lib):
    """32,768 DOFs, shuffled numbering: the FP64 form equals the oracle's
    decisions with operator difference <= 1e-8; the mixed form keeps at
    least 95 % of the ranks and converges within 2 iterations of it."""
    p = inputs.unstructured_operator(64, 64, 8, ratio=1e6, sigma=1.0, seed=5)
    h, ref, depth = setup_pair(hs, oracle_lib, p, 1e-2, threads=8)
    rank_diff(h, ref, depth)
    assert operator_diff(h, ref, p.n, nvec=3) <= 1e-8
    info, rc, xg, res = solve(h, p)
    _, ito, _, rco = ref.pcg(rtol=1e-8)
    assert rc == 0 and rco == 0 and abs(info.iters - ito) <= 1 and res <= 1e-8
    h.close()
    perm, lp, depth = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 4, 0.5)
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_DEVICE, stream=stream(), precision=hs.HS_PREC_MIXED)
    hm = hs.hs_setup(p.n, dev(p.rowptr), dev(p.col), dev(p.val), tree=(perm, lp, depth), opt=opt)
    nd, nt = rank_diff(hm, ref, depth, exact=False)
    info, rc, xg, res = solve(hm, p)
    print(f"unstructured 64x64x8 mixed: ranks differing {nd} of {nt}, PCG {info.iters} vs {ito}, res {res:.2e}")
    assert nd <= 0.05 * nt
    assert rc == 0 and abs(info.iters - ito) <= 2 and res <= 1e-8
    hm.close()


def test_partitioner_option_equals_explicit_tree(hs):
    """hs_setup without a tree and with options.partitioner = multilevel
    builds the tree of hs_partition_multilevel: same levels, ranks and
    phases, and bitwise the same preconditioner output."""
    p = inputs.unstructured_operator(32, 30, 6, ratio=1e5, sigma=1.0, seed=11)
    perm, lp, depth = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 4, 0.5)
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, stream=stream())
    h1 = hs.hs_setup(p.n, p.rowptr, p.col, p.val, tree=(perm, lp, depth), opt=opt)
    opt2 = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, stream=stream(),
                                 partitioner=hs.HS_PART_MULTILEVEL)
    h2 = hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt2)
    assert h1.num_levels() == h2.num_levels() == depth
    for l in range(depth):
        a, b = h1.level_info(l), h2.level_info(l)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    r = dev(np.random.default_rng(2).uniform(-1, 1, p.n))
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    h1.hs_apply(r, z1)
    h2.hs_apply(r, z2)
    torch.cuda.synchronize()
    assert torch.equal(z1, z2)
    h1.close()
    h2.close()


def test_partitioner_option_rejects_unknown_value(hs):
    p = inputs.unstructured_operator(8, 8, 3, ratio=1e3)
    opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, stream=stream(), partitioner=7)
    with pytest.raises(hs.HsError) as e:
        hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt)
    assert e.value.code == hs.HS_ERR_ARG


def test_black_box_solve_256x256x8(hs):
    """524,288 DOFs of a shuffled unstructured mesh, the matrix alone (no
    coordinates, no tree): hs_solve partitions with the multilevel method,
    factors in the mixed form and reaches the true residual 1e-8."""
    p = inputs.unstructured_operator(256, 256, 8, ratio=1e6, sigma=1.0, seed=21)
    x = np.zeros(p.n)
    info, rc = hs.hs_solve(p.n, p.rowptr, p.col, p.val, p.b, x, mem=hs.HS_MEM_HOST, tol=1e-2,
                           precision=hs.HS_PREC_MIXED, partitioner=hs.HS_PART_MULTILEVEL, stream=stream())
    res = np.linalg.norm(p.b - p.matvec(x)) / np.linalg.norm(p.b)
    print(f"black-box 256x256x8: {info.iters} PCG iterations, setup {info.setup_s:.3f} s, "
          f"solve {info.solve_s:.3f} s, residual {res:.2e}")
    assert rc == 0 and info.rel_resid <= 1e-8 and res <= 1e-8
    assert info.iters <= 30

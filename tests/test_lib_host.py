"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
and its host-side partitioner matches the oracle's bit for bit."""
import os
import re

import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def hs():
    from paper_1811_11248_gb300 import build, hsolve
    build.build()
    hsolve.lib()
    return hsolve


def test_exports_every_declared_symbol(hs):
    with open(os.path.join(ROOT, "include", "hsolve.h")) as fh:
        hdr = fh.read()
    declared = set(re.findall(r"^\s*(?:int|const char\*)\s+(hs_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    lib = hs.lib()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(hs.EXPORTED)


def test_default_options_and_status(hs):
    o = hs.hs_default_options()
    assert o.tol == 1e-2 and o.depth == -1 and o.leaf_lines == 4 and o.rtol == 1e-8
    assert hs.lib().hs_status_str(2).decode().startswith("diagonal block")


@pytest.mark.parametrize("use_coords", [True, False])
@pytest.mark.parametrize("make", [
    lambda: inputs.grid_operator(16, 16, 8, ratio=1e4),
    lambda: inputs.grid_operator(12, 10, 5, ratio=1e3, sigma=1.0, bc="ice"),
    lambda: inputs.vector_operator(8, 6, 3, ratio=1e6),
    lambda: inputs.grid_operator(4, 4, 4, ratio=1e-3),
    lambda: inputs.batched_problem(3),
    # 10,000 lines: the top bisections of the coordinate rule on two threads
    lambda: inputs.grid_operator(100, 100, 2, ratio=1e4, sigma=1.0, seed=2, bc="ice"),
])
def test_partition_matches_oracle(hs, oracle_lib, make, use_coords):
    p = make()
    co = np.ascontiguousarray(p.coords) if use_coords else None
    perm, lp, depth = hs.hs_partition_extruded(p.n, p.rowptr, p.col, p.val, co, 4, 0.5)
    operm, olp = oracle_lib.partition(p, 4, use_coords=use_coords)
    assert np.array_equal(perm, operm) and np.array_equal(lp, olp)
    assert depth == oracle_lib.default_depth(len(lp) - 1)


@pytest.mark.parametrize("use_coords", [True, False])
def test_partition_matches_oracle_large(hs, oracle_lib, use_coords):
    """409,600 DOFs in 102,400 lines: large enough for the partitioner's
    parallel line numbering, bisection rounds (with coordinates) and chunked
    leaf permutation."""
    p = inputs.grid_operator(320, 320, 4, ratio=1e4, sigma=1.0, seed=5, bc="ice", shelf=0.5)
    co = np.ascontiguousarray(p.coords) if use_coords else None
    perm, lp, depth = hs.hs_partition_extruded(p.n, p.rowptr, p.col, p.val, co, 4, 0.5)
    operm, olp = oracle_lib.partition(p, 4, use_coords=use_coords)
    assert len(lp) - 1 == 32768
    assert np.array_equal(perm, operm) and np.array_equal(lp, olp)


def _graph_csr(nc, a, b):
    """Symmetric CSR (sorted rows, no self loops) from edge arrays."""
    a, b = np.asarray(a, np.int64), np.asarray(b, np.int64)
    m = a != b
    a, b = np.concatenate([a[m], b[m]]), np.concatenate([b[m], a[m]])
    key = np.unique(a * nc + b)
    rows, cols = key // nc, key % nc
    ptr = np.zeros(nc + 1, np.int64)
    np.add.at(ptr, rows + 1, 1)
    return np.cumsum(ptr), cols.astype(np.int32)


def _grid_graph(nx, ny, diag=False):
    idx = np.arange(nx * ny).reshape(ny, nx)
    a = [idx[:, :-1].ravel(), idx[:-1, :].ravel()]
    b = [idx[:, 1:].ravel(), idx[1:, :].ravel()]
    if diag:
        a.append(idx[:-1, :-1].ravel())
        b.append(idx[1:, 1:].ravel())
    return _graph_csr(nx * ny, np.concatenate(a), np.concatenate(b))


def _random_graph(rng, nc, deg):
    """Random geometric graph in the unit square (about deg neighbours)."""
    pts = rng.random((nc, 2))
    cell = np.sqrt(deg / (np.pi * nc))
    order = np.lexsort(((pts[:, 1] // cell), (pts[:, 0] // cell)))
    a, b = [], []
    grid = {}
    for i in order:
        grid.setdefault((int(pts[i, 0] // cell), int(pts[i, 1] // cell)), []).append(i)
    for (gx, gy), members in grid.items():
        near = [j for dx in (-1, 0, 1) for dy in (-1, 0, 1) for j in grid.get((gx + dx, gy + dy), [])]
        near = np.array(near)
        for i in members:
            d = np.hypot(*(pts[near] - pts[i]).T)
            for j in near[(d < cell) & (near > i)]:
                a.append(i)
                b.append(j)
    return _graph_csr(nc, a, b)


def _compare_plans(hs, oracle_lib, ptr, adj, size0, ranges=None):
    got = hs.hs_plan_level(ptr, adj, size0, ranges)
    ref = oracle_lib.plan_level(ptr, adj, size0)
    for g, r, name in zip(got, ref, ("phase", "vanished", "end_ptr", "end_adj", "all_ptr", "all_adj")):
        assert np.array_equal(g, r), name
    return got


def test_level_plan_matches_oracle_on_a_large_grid(hs, oracle_lib):
    """40,000 clusters: the first phases are large enough for the planner to
    apply their eliminations to the block graph on all threads."""
    ptr, adj = _grid_graph(200, 200)
    size0 = np.random.default_rng(0).integers(1, 6, 200 * 200)
    ph, van = _compare_plans(hs, oracle_lib, ptr, adj, size0)[:2]
    assert ph.max() >= 2 and van.sum() > 0


@pytest.mark.parametrize("nx,ny,diag", [(32, 32, True), (45, 40, False), (64, 32, True)])
def test_level_plan_matches_oracle_bit_planner(hs, oracle_lib, nx, ny, diag):
    """One range of at most 2,048 clusters (the bit-row planner, as at level
    0 of the 64x64x16 workload), planned twice in a row on the same thread so
    that its reused buffers start from the previous plan's contents."""
    ptr, adj = _grid_graph(nx, ny, diag=diag)
    size0 = np.random.default_rng(nx + ny).integers(1, 9, nx * ny)
    first = _compare_plans(hs, oracle_lib, ptr, adj, size0)
    again = _compare_plans(hs, oracle_lib, ptr, adj, size0)
    assert all(np.array_equal(a, b) for a, b in zip(first, again))


def test_level_plan_matches_oracle_on_random_graphs(hs, oracle_lib):
    rng = np.random.default_rng(1)
    for nc, deg in ((3000, 5.0), (20000, 7.0)):
        ptr, adj = _random_graph(rng, nc, deg)
        size0 = rng.integers(1, 9, nc)
        # clusters without blocks may have no DOFs
        isolated = np.flatnonzero(np.diff(ptr) == 0)
        size0[isolated[::2]] = 0
        _compare_plans(hs, oracle_lib, ptr, adj, size0)


def test_level_plan_with_independent_ranges(hs, oracle_lib):
    """Many independent problems, each planned on its own thread: the same
    plan as the whole block-diagonal graph planned at once."""
    rng = np.random.default_rng(2)
    ptrs, adjs, sizes, ranges, base = [], [], [], [], 0
    for k in range(40):
        if k % 3 == 0:
            nx, ny = rng.integers(3, 20, 2)
            ptr, adj = _grid_graph(int(nx), int(ny), diag=bool(k % 2))
        else:
            ptr, adj = _random_graph(rng, int(rng.integers(20, 600)), 6.0)
        nc = len(ptr) - 1
        ptrs.append(ptr[1:] + (adjs and sum(len(x) for x in adjs) or 0))
        adjs.append(adj + base)
        sizes.append(rng.integers(1, 5, nc))
        ranges.append((base, base + nc))
        base += nc
    ptr = np.concatenate([[0]] + ptrs)
    adj = np.concatenate(adjs).astype(np.int32)
    _compare_plans(hs, oracle_lib, ptr, adj, np.concatenate(sizes), np.array(ranges))


def test_level_plan_rejects_bad_input(hs):
    ptr, adj = _grid_graph(3, 3)
    ok = np.ones(9, np.int32)
    hs.hs_plan_level(ptr, adj, ok)
    bad = adj.copy()
    bad[0] = 0  # self loop
    with pytest.raises(hs.HsError):
        hs.hs_plan_level(ptr, bad, ok)
    with pytest.raises(hs.HsError):  # not symmetric
        hs.hs_plan_level(np.array([0, 1, 1]), np.array([1], np.int32), np.ones(2, np.int32))
    with pytest.raises(hs.HsError):  # a block of a cluster without DOFs
        hs.hs_plan_level(ptr, adj, np.where(np.arange(9) == 4, 0, 1))
    with pytest.raises(hs.HsError):  # a block between two ranges
        hs.hs_plan_level(ptr, adj, ok, np.array([[0, 4], [4, 9]]))


def test_partition_rejects_bad_arguments(hs):
    p = inputs.grid_operator(4, 4, 2, ratio=10.0)
    with pytest.raises(hs.HsError):
        hs.hs_partition_extruded(p.n, p.rowptr, p.col, p.val, None, 0, 0.5)


def _partition_in_child(q):
    from paper_1811_11248_gb300 import hsolve as hs2
    p = inputs.anisotropic_64x64x16()
    perm, lp, depth = hs2.hs_partition_extruded(p.n, p.rowptr, p.col, p.val,
                                               np.ascontiguousarray(p.coords), 4, 0.5)
    q.put(int(depth))


def test_host_planner_survives_fork(hs):
    """The planner's worker threads are created on first use; a process
    forked afterwards has none, so its parallel loops must run serially
    instead of waiting for workers that do not exist."""
    import multiprocessing
    p = inputs.anisotropic_64x64x16()
    hs.hs_partition_extruded(p.n, p.rowptr, p.col, p.val, np.ascontiguousarray(p.coords), 4, 0.5)
    ctx = multiprocessing.get_context("fork")
    q = ctx.Queue()
    child = ctx.Process(target=_partition_in_child, args=(q,))
    child.start()
    child.join(timeout=60)
    alive = child.is_alive()
    if alive:
        child.kill()
    assert not alive, "forked child hung in the host planner"
    assert child.exitcode == 0 and q.get(timeout=5) == 8

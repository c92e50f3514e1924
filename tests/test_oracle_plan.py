"""Pins of the oracle's symbolic level plan (the phase rule and the fill
pattern without arithmetic) against hand-worked graphs and against the
phases the numeric oracle takes on a real problem."""
import numpy as np

from oracle import plan_level
from paper_1811_11248_gb300 import inputs


def csr(nc, edges):
    adj = [set() for _ in range(nc)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    ptr = np.zeros(nc + 1, np.int64)
    for c in range(nc):
        ptr[c + 1] = ptr[c] + len(adj[c])
    return ptr, np.array([q for c in range(nc) for q in sorted(adj[c])], np.int32)


def ends(end_ptr, end_adj):
    return [sorted(end_adj[end_ptr[c]:end_ptr[c + 1]].tolist()) for c in range(len(end_ptr) - 1)]


def test_path_of_four():
    """0-1-2-3: phase 0 takes 0 and 2 (both without fill: they leave), which
    couples 1 and 3; 1 then has only that fill block, so it stays (phase 1),
    and 3 follows in phase 2."""
    ptr, adj = csr(4, [(0, 1), (1, 2), (2, 3)])
    ph, van, ep, ea, ap, aa = plan_level(ptr, adj, [2, 2, 2, 2])
    assert ph.tolist() == [0, 1, 0, 2]
    assert van.tolist() == [1, 0, 1, 0]
    assert ends(ep, ea) == [[], [1, 3], [], [1, 3]]
    # every block of the level: the input's, the diagonal and the fill 1-3
    assert ends(ap, aa) == [[0, 1], [0, 1, 2, 3], [1, 2, 3], [1, 2, 3]]


def test_star():
    """Centre 0 with leaves 1-4: the centre goes first and leaves; the leaves
    become a clique of fill blocks and are taken one per phase."""
    ptr, adj = csr(5, [(0, k) for k in range(1, 5)])
    ph, van, ep, ea, ap, aa = plan_level(ptr, adj, [3] * 5)
    assert ph.tolist() == [0, 1, 2, 3, 4]
    assert van.tolist() == [1, 0, 0, 0, 0]
    e = ends(ep, ea)
    assert e[0] == []
    for k in range(1, 5):
        assert e[k] == [1, 2, 3, 4]
    assert ends(ap, aa) == [[0, 1, 2, 3, 4]] * 5


def test_empty_clusters_have_no_phase():
    """1 has no DOFs; 0 leaves first, after which 2 has no block at all (no
    fill), so it leaves too."""
    ptr, adj = csr(3, [(0, 2)])
    ph, van, ep, ea, ap, aa = plan_level(ptr, adj, [1, 0, 1])
    assert ph.tolist() == [0, -1, 1]
    assert van.tolist() == [1, 0, 1]
    assert ends(ep, ea) == [[], [], []]
    assert ends(ap, aa) == [[0, 2], [], [0, 2]]


def test_grid_first_phase_is_the_checkerboard():
    """4-neighbour grid in row-major order: the first phase is the red
    checkerboard (no fill yet, so all of it leaves: plain block Cholesky);
    every black cluster is then coupled to every black cluster that shares
    a red neighbour with it."""
    nx = ny = 6
    idx = lambda i, j: j * nx + i
    edges = [(idx(i, j), idx(i + 1, j)) for j in range(ny) for i in range(nx - 1)]
    edges += [(idx(i, j), idx(i, j + 1)) for j in range(ny - 1) for i in range(nx)]
    ptr, adj = csr(nx * ny, edges)
    ph, van, ep, ea, _, _ = plan_level(ptr, adj, [4] * (nx * ny))
    e = ends(ep, ea)
    nbr = [set(adj[ptr[c]:ptr[c + 1]].tolist()) for c in range(nx * ny)]
    for j in range(ny):
        for i in range(nx):
            c = idx(i, j)
            red = (i + j) % 2 == 0
            assert (ph[c] == 0) == red
            assert bool(van[c]) == red
            if not red:
                assert ph[c] >= 1
                shared = {q for r in nbr[c] for q in nbr[r] if q != c}
                assert shared <= set(e[c]), (c, shared - set(e[c]))
                assert c in e[c]


def test_matches_the_numeric_oracle_phases(oracle_lib):
    """Level 0 of the 16x16x8 ice problem (nonzero ranks): the symbolic plan
    of the level-0 cluster graph gives the numeric oracle's phases, and a
    cluster that leaves the graph has rank 0."""
    p = inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    perm, lp = oracle_lib.partition(p, 4)
    nleaf = len(lp) - 1
    cl = np.empty(p.n, np.int64)
    for c in range(nleaf):
        cl[perm[lp[c]:lp[c + 1]]] = c
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    a, b = cl[rows], cl[p.col]
    m = a != b
    ptr, adj = csr(nleaf, set(zip(a[m].tolist(), b[m].tolist())))
    ph, van = plan_level(ptr, adj, np.diff(lp))[:2]
    f = oracle_lib.Factor(p, perm, lp, 4, 1e-2)
    s0, fin, oph = f.level_info(0)
    assert np.array_equal(ph, oph)
    assert np.all(fin[van == 1] == 0)
    assert fin.max() > 0

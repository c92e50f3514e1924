"""CPU tests of the multilevel partitioner (hs_partition_multilevel): the
column-preserving partition of Sec. 4.2 taken from the matrix alone, with a
graph partitioner in the role the paper gives METIS / Zoltan.

Pins that do not come from the library: lines are found here from the mesh
(DOFs at one horizontal position), the split sizes follow from the
ceil/floor rule, and the first bisection of graphs of at most 20 lines is
compared with the minimum bisection found by enumerating every balanced
split.  The heuristic's cut on larger meshes is compared with the BFS and
coordinate partitions of the same matrix."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hs():
    from paper_1811_11248_gb300 import build, hsolve
    build.build()
    hsolve.lib()
    return hsolve


def lines_of(p):
    """Line id of every DOF: DOFs at one horizontal position."""
    _, line = np.unique(np.round(p.coords, 12), axis=0, return_inverse=True)
    return line.ravel()


def leaf_of(perm, lp, n):
    cl = np.empty(n, np.int64)
    for c in range(len(lp) - 1):
        cl[perm[lp[c]:lp[c + 1]]] = c
    return cl


def line_weights(p, line):
    """Symmetric line-graph weights: sum of |a_ij| between two lines."""
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    k = line.max() + 1
    W = np.zeros((k, k))
    m = line[rows] != line[p.col]
    np.add.at(W, (line[rows[m]], line[p.col[m]]), np.abs(p.val[m]))
    return W


def weighted_cut(p, perm, lp):
    cl = leaf_of(perm, lp, p.n)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    m = cl[rows] != cl[p.col]
    return float(np.abs(p.val[m]).sum()) / 2


CASES = [
    ("grid 16x16x8", lambda: inputs.grid_operator(16, 16, 8, ratio=1e4)),
    ("grid 12x10x5 ice", lambda: inputs.grid_operator(12, 10, 5, ratio=1e3, sigma=1.0, bc="ice")),
    ("vector 8x6x3", lambda: inputs.vector_operator(8, 6, 3, ratio=1e6)),
    ("unstructured 20x17x4", lambda: inputs.unstructured_operator(20, 17, 4, ratio=1e5, sigma=1.0, seed=2)),
    ("unstructured 9x9x3 unshuffled", lambda: inputs.unstructured_operator(9, 9, 3, ratio=1e4, shuffle=False)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("leaf_lines", [1, 4, 7])
def test_lines_whole_and_splits_exact(hs, name, make, leaf_lines):
    p = make()
    perm, lp, depth = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, leaf_lines, 0.5)
    assert np.array_equal(np.sort(perm), np.arange(p.n))
    nleaf = len(lp) - 1
    assert nleaf & (nleaf - 1) == 0
    cl = leaf_of(perm, lp, p.n)
    for c in range(nleaf):
        assert np.all(np.diff(perm[lp[c]:lp[c + 1]]) > 0)  # ascending inside a leaf
    line = lines_of(p)
    nl = line.max() + 1
    leaf_line = np.full(nl, -1)
    for l in range(nl):
        owners = np.unique(cl[line == l])
        assert owners.size == 1, f"line {l} split over leaves {owners}"
        leaf_line[l] = owners[0]
    cnt = np.bincount(leaf_line, minlength=nleaf)
    # 2^L leaves: the fewest levels whose leaves hold at most leaf_lines
    # lines, but never more leaves than lines
    L = nleaf.bit_length() - 1
    assert (1 << L) <= nl
    assert -(-nl // (1 << L)) <= leaf_lines or (1 << (L + 1)) > nl
    assert L == 0 or -(-nl // (1 << (L - 1))) > leaf_lines
    assert cnt.max() == -(-nl // (1 << L)) and cnt.min() == nl // (1 << L)
    # every split of the binary tree: ceil(k/2) lines left, floor(k/2) right
    for d in range(L):
        width = nleaf >> d
        for base in range(0, nleaf, width):
            k = cnt[base:base + width].sum()
            assert cnt[base:base + width // 2].sum() == (k + 1) // 2
    assert depth == max(1 if nleaf >= 2 else 0, L - 2)


def brute_min_bisection(W):
    """Minimum weight of the edges cut by a split into ceil(k/2) / floor(k/2)
    vertices, over every such split (bitmask enumeration, k <= 20)."""
    k = W.shape[0]
    left = (k + 1) // 2
    masks = np.arange(1 << k, dtype=np.int64)
    bits = (masks[:, None] >> np.arange(k)) & 1
    ok = bits.sum(1) == left
    bits = bits[ok].astype(bool)
    iu, ju = np.nonzero(np.triu(W, 1))
    cut = np.zeros(len(bits))
    for i, j in zip(iu, ju):
        cut += W[i, j] * (bits[:, i] != bits[:, j])
    return cut.min()


SMALL = [
    ("grid 4x4", lambda: inputs.grid_operator(4, 4, 3, ratio=1e4)),
    ("grid 2x8", lambda: inputs.grid_operator(2, 8, 3, ratio=1e4)),
    ("chain 1x16", lambda: inputs.grid_operator(1, 16, 3, ratio=1e4)),
    ("grid 4x5 sigma 1", lambda: inputs.grid_operator(4, 5, 3, ratio=1e4, sigma=1.0, seed=2)),
    ("unstructured 5x4 sigma 1", lambda: inputs.unstructured_operator(5, 4, 3, ratio=1e4, sigma=1.0, seed=1)),
    ("unstructured 4x4", lambda: inputs.unstructured_operator(4, 4, 3, ratio=1e4, seed=2)),
    ("unstructured 4x5 sigma 2", lambda: inputs.unstructured_operator(4, 5, 2, ratio=1e4, sigma=2.0, seed=7)),
]


@pytest.mark.parametrize("name,make", SMALL, ids=[c[0] for c in SMALL])
def test_first_bisection_is_a_minimum_bisection(hs, name, make):
    p = make()
    line = lines_of(p)
    W = line_weights(p, line)
    assert np.allclose(W, W.T)
    perm, lp, _ = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 1, 0.5)
    nleaf = len(lp) - 1
    cl = leaf_of(perm, lp, p.n)
    side = np.zeros(W.shape[0], bool)
    for l in range(W.shape[0]):
        side[l] = cl[line == l][0] >= nleaf // 2
    assert (~side).sum() == (W.shape[0] + 1) // 2
    got = W[np.ix_(~side, side)].sum()
    best = brute_min_bisection(W)
    assert got <= best * (1 + 1e-12), (got, best)


@pytest.mark.parametrize("make,geo_factor", [
    (lambda: inputs.grid_operator(64, 64, 4, ratio=1e4, sigma=1.0), 1.15),
    (lambda: inputs.unstructured_operator(40, 40, 6, ratio=1e5, sigma=1.0, seed=3), 1.0),
    (lambda: inputs.unstructured_operator(96, 80, 3, ratio=1e5, seed=4), 1.0),
])
def test_cut_against_bfs_and_coordinates(hs, make, geo_factor):
    """Smaller weighted cut than BFS graph growing on every mesh; on the
    unstructured meshes also smaller than coordinate bisection, and within
    15 % of it on a structured grid (where straight coordinate cuts are
    near optimal)."""
    p = make()
    ml = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 4, 0.5)
    bfs = hs.hs_partition_extruded(p.n, p.rowptr, p.col, p.val, None, 4, 0.5)
    geo = hs.hs_partition_extruded(p.n, p.rowptr, p.col, p.val, np.ascontiguousarray(p.coords), 4, 0.5)
    assert len(ml[1]) == len(bfs[1]) == len(geo[1])
    c_ml, c_bfs, c_geo = (weighted_cut(p, t[0], t[1]) for t in (ml, bfs, geo))
    assert c_ml < c_bfs, (c_ml, c_bfs)
    assert c_ml <= geo_factor * c_geo, (c_ml, c_geo)


_CHILD = """
import hashlib, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_1811_11248_gb300 import hsolve, inputs
p = inputs.unstructured_operator(48, 40, 3, ratio=1e5, sigma=1.0, seed=9)
perm, lp, d = hsolve.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 4, 0.5)
print(hashlib.sha256(perm.tobytes() + lp.tobytes()).hexdigest())
"""


def test_result_does_not_depend_on_thread_count(hs):
    out = []
    for t in ("1", "3", "8"):
        env = dict(os.environ, HS_THREADS=t)
        r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out.append(r.stdout.strip())
    assert out[0] == out[1] == out[2]


def test_shuffled_numbering_finds_the_mesh_lines(hs):
    """With a random DOF numbering the lines are still the mesh's vertical
    lines, and the partition is the same up to that renumbering when the
    line graph is the same (the line ids follow the smallest DOF, so only
    the line count and the leaf sizes are compared)."""
    a = inputs.unstructured_operator(24, 20, 5, ratio=1e5, seed=6, shuffle=False)
    b = inputs.unstructured_operator(24, 20, 5, ratio=1e5, seed=6, shuffle=True)
    for p in (a, b):
        perm, lp, _ = hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 4, 0.5)
        sizes = np.diff(lp)
        assert sizes.sum() == p.n and np.all(sizes % 5 == 0)
        assert len(lp) - 1 == 128 and sizes.max() == 4 * 5


def test_rejects_bad_arguments(hs):
    p = inputs.unstructured_operator(4, 4, 2, ratio=10.0)
    with pytest.raises(hs.HsError):
        hs.hs_partition_multilevel(p.n, p.rowptr, p.col, p.val, 0, 0.5)
    with pytest.raises(hs.HsError):
        hs.hs_partition_multilevel(0, p.rowptr, p.col, p.val, 4, 0.5)

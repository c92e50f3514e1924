"""Pins of the extruded (column-preserving) partitioner, Sec. 4.2."""
import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs


def _check(p, perm, lp, leaf_lines, dofs_per_line):
    n = p.n
    assert np.array_equal(np.sort(perm), np.arange(n))
    nleaf = len(lp) - 1
    assert nleaf & (nleaf - 1) == 0
    cl = np.empty(n, int)
    for c in range(nleaf):
        dofs = perm[lp[c]:lp[c + 1]]
        assert np.all(np.diff(dofs) > 0)  # ascending inside a leaf
        cl[dofs] = c
    # every vertical line (same horizontal position) lies in one cluster
    key = p.coords[:, 0] * 1e6 + p.coords[:, 1]
    for k in np.unique(key):
        assert len(np.unique(cl[key == k])) == 1
    sizes = np.diff(lp) // dofs_per_line
    assert sizes.max() <= leaf_lines and sizes.max() - sizes.min() <= 1
    return cl


@pytest.mark.parametrize("use_coords", [True, False])
@pytest.mark.parametrize("make,dpl", [
    (lambda: inputs.grid_operator(16, 16, 8, ratio=1e4), 8),
    (lambda: inputs.grid_operator(12, 10, 5, ratio=1e3, sigma=1.0, bc="ice"), 5),
    (lambda: inputs.vector_operator(8, 8, 3, ratio=1e6), 6),
])
def test_lines_kept_whole(oracle_lib, make, dpl, use_coords):
    p = make()
    perm, lp = oracle_lib.partition(p, 4, use_coords=use_coords)
    _check(p, perm, lp, 4, dpl)


def test_grid_leaves_are_2x2_columns_and_siblings_adjacent(oracle_lib):
    p = inputs.grid_operator(16, 16, 8, ratio=1e4)
    perm, lp = oracle_lib.partition(p, 4)
    assert len(lp) - 1 == 64
    cl = _check(p, perm, lp, 4, 8)
    for c in range(64):
        xy = p.coords[perm[lp[c]:lp[c + 1]]]
        assert np.ptp(xy[:, 0]) == 1 and np.ptp(xy[:, 1]) == 1
    A = p.dense()
    for c in range(0, 64, 2):
        a = perm[lp[c]:lp[c + 1]]
        b = perm[lp[c + 1]:lp[c + 2]]
        assert np.any(A[np.ix_(a, b)] != 0)


def test_strong_direction_defines_the_lines(oracle_lib):
    """theta = 0.5 test: with horizontal coupling 1000x the vertical one, the
    strongly coupled lines are whole horizontal layers."""
    p = inputs.grid_operator(4, 4, 4, ratio=1e-3)
    perm, lp = oracle_lib.partition(p, 1)
    assert len(lp) - 1 == 4
    k = np.arange(p.n) % 4
    for c in range(4):
        assert len(np.unique(k[perm[lp[c]:lp[c + 1]]])) == 1

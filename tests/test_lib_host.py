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

"""Seeded synthetic inputs: extruded anisotropic diffusion operators.

This module defines the linear systems only. It contains none of the
solver's arithmetic and is the one module that both the CPU oracle and the
CUDA path use.

The paper's test matrices come from the first-order Stokes ice-sheet model on
Antarctic meshes (Sec. 4, Table 2), which are not available.  The stand-ins
have the structure the paper relies on (Sec. 1, Sec. 4.2): an extruded grid of
a few to twenty layers, vertical coupling many orders of magnitude stronger
than horizontal coupling, and clusters that are bundles of vertical lines.

Discretisation (h = 1 in every direction):
  * node (i, j, k) couples to its six face neighbours with -k_face;
  * diagonal = sum of the six face coefficients; faces that leave the grid are
    Dirichlet faces and add to the diagonal only (``neumann_z`` drops the
    top/bottom ones, giving nearly singular column blocks, Sec. 1);
  * node coefficient c = exp(sigma * xi), xi ~ N(0, 1) drawn in DOF order;
    horizontal face = kh * harmonic mean of the two nodes' c; vertical face =
    ratio * that; a Dirichlet face uses the node's own c;
  * DOF index = (j * nx + i) * nz + k (a vertical line is contiguous);
  * right-hand side uniform[-1, 1], drawn from the same generator after xi.
With sigma = 0 the operator is kh*(T_nx + T_ny) + ratio*kh*T_nz in Kronecker
form, whose eigenvalues are sum_d k_d * 4 sin^2(pi m_d / (2 (n_d + 1))) (the
3-D form of the closed form quoted in Sec. 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """A sparse SPD system A x = b in CSR form (both triangles stored)."""

    n: int
    rowptr: np.ndarray  # int64, n + 1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz
    b: np.ndarray  # float64, n
    coords: np.ndarray  # float64, n x 2 horizontal position of each DOF
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.col] = self.val
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        y = np.zeros(self.n)
        np.add.at(y, rows, self.val * x[self.col])
        return y


def _coo_to_csr(n, r, c, v):
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c.astype(np.int32), v.astype(np.float64)


def grid_operator(nx, ny, nz, ratio, sigma=0.0, seed=0, kh=1.0,
                  neumann_z=False, bc="dirichlet", shelf=0.25):
    """Scalar 7-point operator of the module docstring on an nx*ny*nz grid.

    ``bc="ice"`` replaces the top/bottom Dirichlet faces by the ice-sheet
    conditions of Sec. 4.1: homogeneous Neumann on top (k = nz-1) and a Robin
    (basal friction) term on the bottom (k = 0) equal to the Dirichlet face
    times beta(x, y), with beta = 1 on grounded ice and beta = 0 under a
    floating shelf covering the last ``shelf`` fraction of the x range.
    Lateral faces stay Dirichlet.  Shelf columns are then anchored only by
    the weak horizontal coupling: the nearly singular diagonal blocks the
    paper targets (Sec. 1).
    """
    nx, ny, nz = int(nx), int(ny), int(nz)
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    if sigma > 0.0:
        c = np.exp(sigma * rng.standard_normal(n))
    else:
        c = np.ones(n)
    b = rng.uniform(-1.0, 1.0, n)

    idx = np.arange(n, dtype=np.int64)
    k = idx % nz
    ij = idx // nz
    i = ij % nx
    j = ij // nx

    diag = np.zeros(n)
    rows, cols, vals = [], [], []

    def hmean(a, bb):
        return 2.0 * a * bb / (a + bb)

    # (axis mask, neighbour offset, in-grid test, scale)
    faces = [
        (i > 0, -nz, kh),
        (i < nx - 1, +nz, kh),
        (j > 0, -nx * nz, kh),
        (j < ny - 1, +nx * nz, kh),
        (k > 0, -1, kh * ratio),
        (k < nz - 1, +1, kh * ratio),
    ]
    for f, (inside, step, scale) in enumerate(faces):
        src = idx[inside]
        dst = src + step
        coef = scale * hmean(c[src], c[dst])
        rows.append(src)
        cols.append(dst)
        vals.append(-coef)
        np.add.at(diag, src, coef)
        out = idx[~inside]
        if f >= 4 and neumann_z:
            continue
        if f >= 4 and bc == "ice":
            if f == 5:
                continue  # top: natural (Neumann) condition
            grounded = i[out] < nx - int(round(shelf * nx))
            out = out[grounded]  # bottom: Robin, beta = 0 under the shelf
        np.add.at(diag, out, scale * c[out])
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    rowptr, col, val = _coo_to_csr(n, np.concatenate(rows),
                                   np.concatenate(cols), np.concatenate(vals))
    coords = np.stack([i.astype(np.float64), j.astype(np.float64)], axis=1)
    meta = dict(kind="scalar", nx=nx, ny=ny, nz=nz, ratio=float(ratio),
                sigma=float(sigma), seed=int(seed), kh=float(kh),
                neumann_z=bool(neumann_z), bc=bc, shelf=float(shelf),
                dofs_per_node=1)
    return Problem(n, rowptr, col, val, b, coords, meta)


def vector_operator(nx, ny, nz, ratio, coupling=0.5, sigma=0.0, seed=0,
                    bc="dirichlet", shelf=0.25):
    """Two-component operator K (x) [[1, c], [c, 1]], DOFs interleaved per node.

    K is the scalar operator of ``grid_operator``; the 2x2 factor couples the
    two velocity-like components at every stencil entry.  Eigenvalues are
    (1 - c) and (1 + c) times those of K, so the operator is SPD for |c| < 1.
    """
    k = grid_operator(nx, ny, nz, ratio, sigma=sigma, seed=seed, bc=bc,
                      shelf=shelf)
    n = 2 * k.n
    rows_k = np.repeat(np.arange(k.n, dtype=np.int64), np.diff(k.rowptr))
    blk = np.array([[1.0, coupling], [coupling, 1.0]])
    rr, cc, vv = [], [], []
    for a in range(2):
        for bb in range(2):
            rr.append(2 * rows_k + a)
            cc.append(2 * k.col.astype(np.int64) + bb)
            vv.append(k.val * blk[a, bb])
    rowptr, col, val = _coo_to_csr(n, np.concatenate(rr), np.concatenate(cc),
                                   np.concatenate(vv))
    rng = np.random.default_rng(seed + 1_000_003)
    b = rng.uniform(-1.0, 1.0, n)
    coords = np.repeat(k.coords, 2, axis=0)
    meta = dict(k.meta)
    meta.update(kind="vector", coupling=float(coupling), dofs_per_node=2)
    return Problem(n, rowptr, col, val, b, coords, meta)


def unstructured_operator(mx, my, nz, ratio, sigma=0.0, seed=0, kh=1.0, bc="ice",
                          shelf=0.25, jitter=0.4, grade=0.5, shuffle=True):
    """Extruded operator on an unstructured horizontal mesh (Sec. 4: the
    ice-sheet meshes are unstructured triangulations extruded in layers).

    Horizontal mesh: the mx*my points of a unit lattice, each moved by
    uniform[-jitter, jitter] in x and y, then graded in x by
    x <- x - grade * (L/2pi) sin(2pi x/L) (L = mx - 1; the points crowd
    around x = 0 and x = L and thin out in between), and joined by their
    Delaunay triangulation (scipy.spatial).  Each triangle edge (u, v) of
    length l couples the two nodes with kh * hmean(c_u, c_v) / l in every
    layer; the outermost ring of lattice points carries a lateral Dirichlet
    term kh * c.  Layers, vertical coupling (ratio), node coefficients
    c = exp(sigma * xi) and the bottom/top conditions are those of
    ``grid_operator`` (bc "ice": Neumann top, Robin bottom with beta = 0 for
    x >= (1 - shelf) * L).  Unshuffled DOF index = node * nz + k;
    ``shuffle`` renumbers the DOFs by a seeded random permutation, so that
    neither the lines nor the mesh can be read off the numbering (the
    partitioner then has only the matrix).  xi, then b, are drawn in the
    unshuffled order from the seeded generator, the permutation after them.
    """
    from scipy.spatial import Delaunay

    mx, my, nz = int(mx), int(my), int(nz)
    nn = mx * my
    n = nn * nz
    rng = np.random.default_rng(seed)
    c = np.exp(sigma * rng.standard_normal(n)) if sigma > 0.0 else np.ones(n)
    b = rng.uniform(-1.0, 1.0, n)
    gi, gj = np.meshgrid(np.arange(mx, dtype=np.float64), np.arange(my, dtype=np.float64))
    gi, gj = gi.ravel(), gj.ravel()  # node = j * mx + i
    prng = np.random.default_rng(seed + 500_009)
    px = gi + prng.uniform(-jitter, jitter, nn)
    py = gj + prng.uniform(-jitter, jitter, nn)
    span = max(mx - 1, 1)
    px = px - grade * span / (2 * np.pi) * np.sin(2 * np.pi * px / span)
    tri = Delaunay(np.stack([px, py], axis=1)).simplices.astype(np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)  # undirected edges u < v
    length = np.hypot(px[e[:, 0]] - px[e[:, 1]], py[e[:, 0]] - py[e[:, 1]])
    ring = (gi == 0) | (gi == mx - 1) | (gj == 0) | (gj == my - 1)

    def hmean(a, bb):
        return 2.0 * a * bb / (a + bb)

    kk = np.arange(nz, dtype=np.int64)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    # horizontal edges in every layer
    su = (e[:, 0][:, None] * nz + kk[None, :]).ravel()
    sv = (e[:, 1][:, None] * nz + kk[None, :]).ravel()
    coef = kh * hmean(c[su], c[sv]) / np.repeat(length, nz)
    for src, dst in ((su, sv), (sv, su)):
        rows.append(src)
        cols.append(dst)
        vals.append(-coef)
        np.add.at(diag, src, coef)
    lat = (np.flatnonzero(ring)[:, None] * nz + kk[None, :]).ravel()
    np.add.at(diag, lat, kh * c[lat])
    # vertical couplings and the bottom/top conditions
    idx = np.arange(n, dtype=np.int64)
    k = idx % nz
    node = idx // nz
    for inside, step in ((k > 0, -1), (k < nz - 1, +1)):
        src = idx[inside]
        dst = src + step
        cv = kh * ratio * hmean(c[src], c[dst])
        rows.append(src)
        cols.append(dst)
        vals.append(-cv)
        np.add.at(diag, src, cv)
    bottom, top = idx[k == 0], idx[k == nz - 1]
    if bc == "ice":
        bottom = bottom[px[node[bottom]] < (1.0 - shelf) * span]
        np.add.at(diag, bottom, kh * ratio * c[bottom])
    else:
        for out in (bottom, top):
            np.add.at(diag, out, kh * ratio * c[out])
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    r = np.concatenate(rows)
    cc = np.concatenate(cols)
    coords = np.stack([px[node], py[node]], axis=1)
    if shuffle:
        q = np.random.default_rng(seed + 900_001).permutation(n)  # old DOF i -> new q[i]
        r, cc = q[r], q[cc]
        bn = np.empty(n)
        bn[q] = b
        b = bn
        cn = np.empty_like(coords)
        cn[q] = coords
        coords = cn
    rowptr, col, val = _coo_to_csr(n, r, cc, np.concatenate(vals))
    meta = dict(kind="unstructured", mx=mx, my=my, nz=nz, nodes=nn, edges=int(len(e)),
                ratio=float(ratio), sigma=float(sigma), seed=int(seed), kh=float(kh), bc=bc,
                shelf=float(shelf), jitter=float(jitter), grade=float(grade), shuffle=bool(shuffle),
                dofs_per_node=1)
    return Problem(n, rowptr, col, val, b, coords, meta)


# ---------------------------------------------------------------------------
# The named workloads (sizes and seeds fixed here, one place).
# ---------------------------------------------------------------------------

def anisotropic_16x16x8():
    """16x16x8 (N = 2048), kh = 1, kv = 1e4, constant coefficients, seed 0.

    64 leaf clusters of 2x2 vertical lines (32 DOFs), 4 elimination levels,
    tolerance 1e-2.
    """
    p = grid_operator(16, 16, 8, ratio=1e4, sigma=0.0, seed=0)
    p.meta.update(name="aniso-16x16x8", leaf_lines=4, depth=4, tol=1e-2)
    return p


ICE_SHELF = 0.5  # fraction of the x range under a floating shelf


def anisotropic_64x64x16(sigma=1.0, seed=1):
    """64x64x16 (N = 65,536), ratio 1e6, log-normal kh (sigma 1, seed 1).

    Ice-sheet boundary conditions (Neumann top, Robin bottom, shelf on half
    the domain).  1024 leaf clusters of 2x2 lines (64 DOFs), 8 levels.
    """
    p = grid_operator(64, 64, 16, ratio=1e6, sigma=sigma, seed=seed,
                      bc="ice", shelf=ICE_SHELF)
    p.meta.update(name="aniso-64x64x16", leaf_lines=4, depth=8, tol=1e-2)
    return p


def batched_problem(p):
    """Problem p (0..255) of the batched workload.

    Grid nx, ny even in [16, 48], nz in [4, 12], ratio 10^U[3, 6],
    horizontal coefficient 1; all draws from default_rng(p), the
    right-hand side drawn after the shape.
    """
    rng = np.random.default_rng(p)
    nx = 2 * int(rng.integers(8, 25))
    ny = 2 * int(rng.integers(8, 25))
    nz = int(rng.integers(4, 13))
    ratio = float(10.0 ** rng.uniform(3.0, 6.0))
    prob = grid_operator(nx, ny, nz, ratio=ratio, sigma=0.0, seed=0,
                         bc="ice", shelf=ICE_SHELF)
    prob.b = rng.uniform(-1.0, 1.0, prob.n)
    prob.meta.update(name=f"batched-{p}", leaf_lines=4, depth=None, tol=1e-2,
                     seed=int(p))
    return prob


def thin_shell_vector(nx=256, ny=256, nz=10):
    """Two-component thin-shell operator, ratio 1e6, coupling 0.5."""
    p = vector_operator(nx, ny, nz, ratio=1e6, coupling=0.5, bc="ice",
                        shelf=ICE_SHELF)
    p.meta.update(name=f"vector-{nx}x{ny}x{nz}x2", leaf_lines=4, depth=None,
                  tol=1e-2)
    return p


def anisotropic_512x512x20():
    """512x512x20 (N = 5,242,880), ratio 1e6, log-normal kh (sigma 1.5)."""
    p = grid_operator(512, 512, 20, ratio=1e6, sigma=1.5, seed=5, bc="ice",
                      shelf=ICE_SHELF)
    p.meta.update(name="aniso-512x512x20", leaf_lines=4, depth=None, tol=1e-2)
    return p


def closed_form_eigenvalues(nx, ny, nz, ratio, kh=1.0):
    """Eigenvalues of the constant-coefficient Dirichlet operator (sorted)."""
    def lam(n):
        m = np.arange(1, n + 1)
        return 4.0 * np.sin(np.pi * m / (2.0 * (n + 1))) ** 2
    e = (kh * lam(nx)[:, None, None] + kh * lam(ny)[None, :, None]
         + kh * ratio * lam(nz)[None, None, :])
    return np.sort(e.ravel())


def block_diagonal(problems):
    """Stack independent problems into one block-diagonal system.

    Returns (prob_ptr int64[len + 1], Problem): problem p owns rows and
    columns prob_ptr[p] .. prob_ptr[p + 1]; b and coords are concatenated.
    """
    pp = np.zeros(len(problems) + 1, np.int64)
    for k, q in enumerate(problems):
        pp[k + 1] = pp[k] + q.n
    rp = [np.zeros(1, np.int64)]
    nz = 0
    for q in problems:
        rp.append(q.rowptr[1:] + nz)
        nz += q.nnz
    col = np.concatenate([q.col.astype(np.int64) + pp[k]
                          for k, q in enumerate(problems)]).astype(np.int32)
    out = Problem(n=int(pp[-1]), rowptr=np.concatenate(rp),
                  col=col, val=np.concatenate([q.val for q in problems]),
                  b=np.concatenate([q.b for q in problems]),
                  coords=np.concatenate([q.coords for q in problems]),
                  meta=dict(name=f"batch-{len(problems)}"))
    return pp, out


def batched_workload(count=256):
    """The first `count` problems of the batched workload, stacked."""
    return block_diagonal([batched_problem(p) for p in range(count)])


def mlp_init_params(seed, nin=8, nh=64):
    """Seeded initial weights of the rank predictor (He-style normal weights,
    zero biases) in its flat layout W1 (nh x nin), b1, W2 (nh x nh), b2, w3, b3."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal(nh * nin) * np.sqrt(2.0 / nin), np.zeros(nh),
             rng.standard_normal(nh * nh) * np.sqrt(2.0 / nh), np.zeros(nh),
             rng.standard_normal(nh) * np.sqrt(1.0 / nh), np.zeros(1)]
    return np.concatenate(parts)


def mlp_batch_order(n, batch, epochs, seed):
    """Sample order of minibatch training: one seeded permutation of the n
    samples per epoch, cut into full batches (a ragged tail is dropped)."""
    rng = np.random.default_rng(seed)
    steps = n // batch
    return np.concatenate([rng.permutation(n)[:steps * batch] for _ in range(epochs)]).astype(np.int32)

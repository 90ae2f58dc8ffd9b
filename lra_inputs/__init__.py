"""Seeded synthetic inputs for C-A CUR low-rank approximation.

This module only draws data: matrices, point sets, initial index sets,
multiplier descriptors and sample positions.  It holds none of the method's
arithmetic, so both the FP64 oracle (``oracle/``) and the CUDA library take
their inputs from here without sharing any computation.

The random choices the method itself makes -- the initial row set I0 of the
Tests 2 schedule, the random diagonal D and permutation P of the abridged
randomized Hadamard multiplier D H_{n,d} P, the positions and signs of the
sparse +-1 multiplier, the rows and columns of the a-posteriori residual
sample -- are drawn here too and passed to both sides as plain arrays.

Workload recipes (numpy PCG64 ``default_rng(seed)``):

* ``dense_lowrank``  -- A = U diag(s) V^T + noise * G, U, V from QR of Gaussians
  (the 256 x 256, rank-8, s_i = 2^-i, 1e-8 noise case and its noiseless variant).
* ``factor_gaussian`` -- W = G1 G2 + eps G3, the paper's random test matrices.
* ``dense_spiky`` -- A = G1 diag(2^{-i/2}) G2 + 1e-6 G in FP32, with 1% of entries
  replaced by +-10 spikes (8192 x 8192, numerical rank 32).
* ``laplace_clusters`` -- targets in [0,1]^3 and sources in [3,4]x[0,1]^2.
* ``fmm_blocks`` -- octree over uniform points in [0,1]^3, interaction-list
  block pairs (well-separated boxes), Morton-sorted points so that every box is
  a contiguous index range.
* ``gaussian_blocks`` -- target / source clouds in separated unit cubes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SRC_DENSE, SRC_LAPLACE, SRC_GAUSSIAN = 0, 1, 2
MULT_NONE, MULT_ARHT, MULT_SPARSE, MULT_BIDIAG, MULT_ARFT = 0, 1, 2, 3, 4


@dataclass
class Problem:
    """An m x n input: a dense row-major array or a kernel on two point sets,
    optionally with a right multiplier descriptor (data only)."""

    src: int
    m: int
    n: int
    W: Optional[np.ndarray] = None          # dense (m, n) float64 or float32, C-contiguous
    X: Optional[np.ndarray] = None          # (m, 3) float64 target points
    Y: Optional[np.ndarray] = None          # (n, 3) float64 source points
    ell: float = 1.0                        # Gaussian length scale
    mkind: int = MULT_NONE
    depth: int = 0                          # ARHT recursion depth d (bidiagonal: number of factors q)
    perm: Optional[np.ndarray] = None       # ARHT permutation (n,) int32 (bidiagonal: (q, n) permutations)
    dsign: Optional[np.ndarray] = None      # ARHT diagonal (n,) int8, +-1 (bidiagonal: (q, n) signs)
    nnz: int = 0                            # sparse multiplier nonzeros per column
    srow: Optional[np.ndarray] = None       # (n, nnz) int32 ascending per column
    ssign: Optional[np.ndarray] = None      # (n, nnz) int8, +-1
    entries: str = "f64"                    # kernel: entries evaluated in "f64", "f32" or "bf16" (Laplace)
    mside: int = 0                          # multiplier side: 0 right (W M, M n x n), 1 left (M^T W, M m x m)
    dcplx: Optional[np.ndarray] = None      # ARFT diagonal D: (n, 2) float64 (real, imaginary), |D_r| = 1
    meta: dict = field(default_factory=dict)

    @property
    def dtype(self) -> str:
        if self.W is None:
            return self.entries
        return "f32" if self.W.dtype == np.float32 else "f64"


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- index sets
def initial_rows(m: int, k: int, seed: int) -> np.ndarray:
    """I0: the first k entries of a seeded random permutation of range(m)."""
    return rng(seed).permutation(m)[:k].astype(np.int32)


def sample_positions(m: int, n: int, q: int, s: int, seed: int):
    """q distinct rows and s distinct columns, uniformly without replacement."""
    g = rng(seed)
    Q = g.choice(m, size=q, replace=False).astype(np.int32)
    S = g.choice(n, size=s, replace=False).astype(np.int32)
    return Q, S


# ---------------------------------------------------------------- multipliers
def arht_descriptor(n: int, depth: int, seed: int):
    """Random diagonal D (Rademacher +-1) and permutation P for D H_{n,d} P."""
    if depth < 1 or n % (1 << depth) != 0:
        raise ValueError("n must be a multiple of 2^depth, depth >= 1")
    g = rng(seed)
    perm = g.permutation(n).astype(np.int32)
    dsign = np.where(g.random(n) < 0.5, -1, 1).astype(np.int8)
    return perm, dsign


def sparse_pm1_descriptor(n: int, nnz: int, seed: int):
    """nnz distinct rows per column (sorted ascending) with random signs."""
    g = rng(seed)
    srow = np.empty((n, nnz), dtype=np.int32)
    for j in range(n):
        srow[j] = np.sort(g.choice(n, size=nnz, replace=False))
    ssign = np.where(g.random((n, nnz)) < 0.5, -1, 1).astype(np.int8)
    return srow, ssign


def gaussian_sketch(n: int, k: int, seed: int) -> np.ndarray:
    """An n x k Gaussian matrix (FP64, standard normal): the Hbar of the
    Gaussian-sampling CUR."""
    return np.ascontiguousarray(rng(seed).standard_normal((n, k)))


def bidiag_descriptor(n: int, q: int, seed: int):
    """q factors (I + D_i S) P_i: per factor a random permutation (column a of P_i
    is e_{perm[i, a]}) and Rademacher signs D_i (q x n each)."""
    if q < 1 or n < 2:
        raise ValueError("q >= 1 factors, n >= 2")
    g = rng(seed)
    perms = np.stack([g.permutation(n) for _ in range(q)]).astype(np.int32)
    signs = np.where(g.random((q, n)) < 0.5, -1, 1).astype(np.int8)
    return perms, signs


def _side(p: Problem, side: str):
    """(order of M, mside) for a multiplier on the given side of p."""
    if side not in ("right", "left"):
        raise ValueError("side is 'right' or 'left'")
    return (p.n, 0) if side == "right" else (p.m, 1)


def with_bidiag(p: Problem, q: int, seed: int, side: str = "right") -> Problem:
    order, p.mside = _side(p, side)
    perms, signs = bidiag_descriptor(order, q, seed)
    p.mkind, p.depth, p.perm, p.dsign = MULT_BIDIAG, q, perms, signs
    return p


def with_arht(p: Problem, depth: int, seed: int, side: str = "right") -> Problem:
    order, p.mside = _side(p, side)
    perm, dsign = arht_descriptor(order, depth, seed)
    p.mkind, p.depth, p.perm, p.dsign = MULT_ARHT, depth, perm, dsign
    return p


def arft_descriptor(n: int, depth: int, seed: int):
    """Random permutation P and diagonal D uniform on the complex unit circle for
    D Omega_{n,d} P: D_r = exp(2 pi sqrt(-1) u_r), u_r uniform in [0, 1), stored
    as (cos, sin) pairs."""
    if depth < 1 or n % (1 << depth) != 0:
        raise ValueError("n must be a multiple of 2^depth, depth >= 1")
    g = rng(seed)
    perm = g.permutation(n).astype(np.int32)
    ang = 2.0 * np.pi * g.random(n)
    return perm, np.ascontiguousarray(np.stack([np.cos(ang), np.sin(ang)], axis=1))


def with_arft(p: Problem, depth: int, seed: int) -> Problem:
    """Right abridged randomized Fourier multiplier in real form: W' = W [Re M, Im M]
    (2n columns), M = 2^{-d/2} D Omega_{n,d} P."""
    perm, dc = arft_descriptor(p.n, depth, seed)
    p.mkind, p.depth, p.perm, p.dcplx, p.mside = MULT_ARFT, depth, perm, dc, 0
    return p


def with_sparse(p: Problem, nnz: int, seed: int, side: str = "right") -> Problem:
    order, p.mside = _side(p, side)
    srow, ssign = sparse_pm1_descriptor(order, nnz, seed)
    p.mkind, p.nnz, p.srow, p.ssign = MULT_SPARSE, nnz, srow, ssign
    return p


# ---------------------------------------------------------------- dense inputs
def dense_lowrank(m: int = 256, n: int = 256, r: int = 8, noise: float = 1e-8, seed: int = 0) -> Problem:
    """A = U diag(2^-1 .. 2^-r) V^T + noise * G, U and V from QR of Gaussians."""
    g = rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((m, r)))
    V, _ = np.linalg.qr(g.standard_normal((n, r)))
    s = 2.0 ** -np.arange(1, r + 1)
    A = (U * s) @ V.T
    if noise:
        A = A + noise * g.standard_normal((m, n))
    return Problem(SRC_DENSE, m, n, W=np.ascontiguousarray(A), meta={"rank": r, "s": s})


def factor_gaussian(n: int = 256, r: int = 8, eps: float = 1e-10, seed: int = 0) -> Problem:
    """W = G1 G2 + eps G3 (G1 n x r, G2 r x n, G3 n x n Gaussian)."""
    g = rng(seed)
    W = g.standard_normal((n, r)) @ g.standard_normal((r, n)) + eps * g.standard_normal((n, n))
    return Problem(SRC_DENSE, n, n, W=np.ascontiguousarray(W), meta={"rank": r})


def dense_spiky(n: int = 8192, r: int = 32, noise: float = 1e-6, spike_frac: float = 0.01,
                spike: float = 10.0, seed: int = 0) -> Problem:
    """FP32 W = G1 diag(2^{-i/2}) G2 + noise G, then a fraction of the entries
    (uniform positions without replacement) replaced by +-spike."""
    g = rng(seed)
    G1 = g.standard_normal((n, r), dtype=np.float32)
    G2 = g.standard_normal((r, n), dtype=np.float32)
    s = (2.0 ** (-np.arange(1, r + 1) / 2.0)).astype(np.float32)
    W = (G1 * s) @ G2
    W += np.float32(noise) * g.standard_normal((n, n), dtype=np.float32)
    nsp = int(round(spike_frac * n * n))
    if nsp:
        pos = g.choice(n * n, size=nsp, replace=False)
        sg = np.where(g.random(nsp) < 0.5, -spike, spike).astype(np.float32)
        W.reshape(-1)[pos] = sg
    return Problem(SRC_DENSE, n, n, W=np.ascontiguousarray(W, dtype=np.float32), meta={"rank": r})


# ---------------------------------------------------------------- kernel inputs
def laplace_clusters(m: int = 65536, n: int = 65536, offset: float = 3.0, seed: int = 0) -> Problem:
    """Targets uniform in [0,1]^3, sources uniform in [offset, offset+1] x [0,1]^2;
    entries 1/|x - y| evaluated on demand."""
    g = rng(seed)
    X = g.random((m, 3))
    Y = g.random((n, 3))
    Y[:, 0] += offset
    return Problem(SRC_LAPLACE, m, n, X=np.ascontiguousarray(X), Y=np.ascontiguousarray(Y))


def gaussian_clusters(m: int = 1024, n: int = 1024, ell: float = 0.3, offset: float = 2.0,
                      seed: int = 0) -> Problem:
    """Targets in [0,1]^3, sources in [offset, offset+1] x [0,1]^2;
    entries exp(-|x - y|^2 / (2 ell^2))."""
    g = rng(seed)
    X = g.random((m, 3))
    Y = g.random((n, 3))
    Y[:, 0] += offset
    return Problem(SRC_GAUSSIAN, m, n, X=np.ascontiguousarray(X), Y=np.ascontiguousarray(Y), ell=ell)


def hmt11_laplacian(n: int = 1024, nodes: int = 8) -> Problem:
    """The discretised single-layer Laplacian of the bidiagonal pre-processing
    tests (input matrices (i), replicated from [HMT11, Section 7.1]): targets
    x_i = 2 w^i on the circle of radius 2 (w = exp(2 pi sqrt(-1) / n)), sources
    the arcs of the unit circle between the angles 2 pi j / n and 2 pi (j+1) / n,
    and w_ij = psi * integral over arc j of log|x_i - y| dy.  Since
    |2 e^{i t} - e^{i f}|^2 = 5 - 4 cos(t - f), each arc integral is taken by
    ``nodes``-point Gauss-Legendre quadrature of 0.5 log(5 - 4 cos(t - f)); the
    entry depends on (i - j) mod n only, so W is built circulant.  psi =
    1 / (2 pi ln 2) makes ||W|| = 1: the mean of log|x - y| over the unit circle
    is log|x| = ln 2, the largest eigenvalue.  Dense FP64, n x n."""
    t, wq = np.polynomial.legendre.leggauss(nodes)
    psi = 1.0 / (2.0 * np.pi * np.log(2.0))
    d = np.arange(n, dtype=np.float64)
    # angle between target i and the quadrature points of arc j, for d = i - j
    ang = 2.0 * np.pi * (d[:, None] - 0.5 * (1.0 + t[None, :])) / n
    c = psi * (np.pi / n) * (0.5 * np.log(5.0 - 4.0 * np.cos(ang)) @ wq)
    i = np.arange(n)
    W = c[(i[:, None] - i[None, :]) % n]
    return Problem(SRC_DENSE, n, n, W=np.ascontiguousarray(W), meta={"psi": psi})


def _morton3(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray, bits: int) -> np.ndarray:
    code = np.zeros(ix.shape, dtype=np.int64)
    for b in range(bits):
        code |= ((ix >> b) & 1).astype(np.int64) << (3 * b + 2)
        code |= ((iy >> b) & 1).astype(np.int64) << (3 * b + 1)
        code |= ((iz >> b) & 1).astype(np.int64) << (3 * b)
    return code


def fmm_blocks(npts: int = 1 << 20, leaf: int = 64, min_size: int = 64, max_size: int = 2048,
               nblocks: int = 4096, seed: int = 0):
    """Octree over npts uniform points in [0,1]^3 and its well-separated block pairs.

    The tree is refined uniformly to the first level whose boxes hold at most
    ``leaf`` points on average.  Points are sorted by the Morton code of their
    finest-level box, so every box at every level is a contiguous index range.
    The interaction list of a box is the set of children of its parent's
    neighbours that are not its own neighbours (neighbours: boxes touching it,
    diagonals included).  Block pairs (target box, source box) are taken from
    every level at which both boxes hold between ``min_size`` and ``max_size``
    points; a seeded subset of ``nblocks`` pairs is kept, sorted by level.

    Returns (Problem over the sorted points with X = Y, blocks int64 (nb, 4) =
    (row0, nrows, col0, ncols), levels int32 (nb,)).
    """
    g = rng(seed)
    P = g.random((npts, 3))
    L = 1
    while npts / (8 ** L) > leaf:
        L += 1
    side = 1 << L
    ijk = np.minimum((P * side).astype(np.int64), side - 1)
    code = _morton3(ijk[:, 0], ijk[:, 1], ijk[:, 2], L)
    order = np.argsort(code, kind="stable")
    P = np.ascontiguousarray(P[order])
    code = code[order]
    pairs = []
    for lev in range(2, L + 1):
        shift = 3 * (L - lev)
        bcode = code >> shift
        nb_side = 1 << lev
        starts = np.searchsorted(bcode, np.arange(8 ** lev), side="left")
        ends = np.searchsorted(bcode, np.arange(8 ** lev), side="right")
        counts = ends - starts
        # box coordinates for each Morton code at this level
        codes = np.arange(8 ** lev, dtype=np.int64)
        bx = np.zeros_like(codes); by = np.zeros_like(codes); bz = np.zeros_like(codes)
        for b in range(lev):
            bx |= ((codes >> (3 * b + 2)) & 1) << b
            by |= ((codes >> (3 * b + 1)) & 1) << b
            bz |= ((codes >> (3 * b)) & 1) << b
        coord_to_code = np.empty((nb_side, nb_side, nb_side), dtype=np.int64)
        coord_to_code[bx, by, bz] = codes
        ok = (counts >= min_size) & (counts <= max_size)
        if not ok.any():
            continue
        for c in np.nonzero(ok)[0]:
            x, y, z = bx[c], by[c], bz[c]
            px, py, pz = x >> 1, y >> 1, z >> 1
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        qx, qy, qz = px + dx, py + dy, pz + dz
                        if not (0 <= qx < nb_side // 2 and 0 <= qy < nb_side // 2 and 0 <= qz < nb_side // 2):
                            continue
                        for cx in (0, 1):
                            for cy in (0, 1):
                                for cz in (0, 1):
                                    sx, sy, sz = 2 * qx + cx, 2 * qy + cy, 2 * qz + cz
                                    if max(abs(sx - x), abs(sy - y), abs(sz - z)) <= 1:
                                        continue
                                    sc = coord_to_code[sx, sy, sz]
                                    if not ok[sc]:
                                        continue
                                    pairs.append((starts[c], counts[c], starts[sc], counts[sc], lev))
    pairs = np.asarray(pairs, dtype=np.int64)
    if len(pairs) > nblocks:
        sel = np.sort(g.choice(len(pairs), size=nblocks, replace=False))
        pairs = pairs[sel]
    blocks = np.ascontiguousarray(pairs[:, :4])
    levels = pairs[:, 4].astype(np.int32)
    prob = Problem(SRC_LAPLACE, npts, npts, X=P, Y=P, meta={"levels": L})
    return prob, blocks, levels


def _pieces(start: int, count: int, max_len):
    """[start, start + count) as consecutive pieces of at most max_len (nearly equal)."""
    if max_len is None or count <= max_len:
        return [(start, count)]
    npc = -(-count // max_len)
    base, extra = divmod(count, npc)
    out, o = [], start
    for i in range(npc):
        sz = base + (1 if i < extra else 0)
        out.append((o, sz))
        o += sz
    return out


def fmm_partition(npts: int = 1 << 16, leaf: int = 128, seed: int = 0, max_block=None):
    """The complete far/near partition of the Laplace matrix K(P, P) over npts
    uniform points in [0,1]^3 (the octree and interaction lists of fmm_blocks,
    every level, no sampling): the points sorted by the Morton code of their
    finest box; far blocks (target box, source box) from the interaction lists
    of every level 2..L (children of the parent's neighbours that do not touch
    the box); near blocks (leaf, leaf) for touching leaves, the leaf itself
    included.  Together the blocks cover every (i, j) exactly once (the diagonal
    i = j lies in the near field).  Empty boxes are skipped.

    Returns (Problem over the sorted points, far int64 (nf, 6) = (row0, nrows,
    col0, ncols, level, target box), near int64 (nn, 5) = (row0, nrows, col0,
    ncols, target leaf), levels L).  Far blocks are ordered by level, then
    target box, then source box; near blocks by target leaf, then source leaf.

    max_block (optional): far blocks with more rows or columns than this are cut
    into nearly equal row and column pieces (a sub-block of a well-separated
    pair is still well separated, and the pieces cover the block once); a row
    piece becomes a target of its own, with the id 64 box + piece."""
    g = rng(seed)
    P = g.random((npts, 3))
    L = 1
    while npts / (8 ** L) > leaf:
        L += 1
    side = 1 << L
    ijk = np.minimum((P * side).astype(np.int64), side - 1)
    code = _morton3(ijk[:, 0], ijk[:, 1], ijk[:, 2], L)
    order = np.argsort(code, kind="stable")
    P = np.ascontiguousarray(P[order])
    code = code[order]

    def level_boxes(lev):
        shift = 3 * (L - lev)
        bcode = code >> shift
        nbox = 8 ** lev
        starts = np.searchsorted(bcode, np.arange(nbox), side="left")
        counts = np.searchsorted(bcode, np.arange(nbox), side="right") - starts
        codes = np.arange(nbox, dtype=np.int64)
        bx = np.zeros_like(codes); by = np.zeros_like(codes); bz = np.zeros_like(codes)
        for b in range(lev):
            bx |= ((codes >> (3 * b + 2)) & 1) << b
            by |= ((codes >> (3 * b + 1)) & 1) << b
            bz |= ((codes >> (3 * b)) & 1) << b
        n = 1 << lev
        c2c = np.empty((n, n, n), dtype=np.int64)
        c2c[bx, by, bz] = codes
        return starts, counts, bx, by, bz, c2c

    far = []
    for lev in range(2, L + 1):
        starts, counts, bx, by, bz, c2c = level_boxes(lev)
        n = 1 << lev
        for c in range(8 ** lev):
            if counts[c] == 0:
                continue
            x, y, z = bx[c], by[c], bz[c]
            srcs = []
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        qx, qy, qz = (x >> 1) + dx, (y >> 1) + dy, (z >> 1) + dz
                        if not (0 <= qx < n // 2 and 0 <= qy < n // 2 and 0 <= qz < n // 2):
                            continue
                        for cx in (0, 1):
                            for cy in (0, 1):
                                for cz in (0, 1):
                                    sx, sy, sz = 2 * qx + cx, 2 * qy + cy, 2 * qz + cz
                                    if max(abs(sx - x), abs(sy - y), abs(sz - z)) <= 1:
                                        continue
                                    sc = c2c[sx, sy, sz]
                                    if counts[sc] > 0:
                                        srcs.append(int(sc))
            if max_block is None:
                for sc in sorted(srcs):
                    far.append((starts[c], counts[c], starts[sc], counts[sc], lev, c))
            else:
                for pi, (r0, nr) in enumerate(_pieces(int(starts[c]), int(counts[c]), max_block)):
                    for sc in sorted(srcs):
                        for c0, nc in _pieces(int(starts[sc]), int(counts[sc]), max_block):
                            far.append((r0, nr, c0, nc, lev, 64 * c + pi))
    starts, counts, bx, by, bz, c2c = level_boxes(L)
    n = 1 << L
    near = []
    for c in range(8 ** L):
        if counts[c] == 0:
            continue
        x, y, z = bx[c], by[c], bz[c]
        srcs = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    sx, sy, sz = x + dx, y + dy, z + dz
                    if 0 <= sx < n and 0 <= sy < n and 0 <= sz < n and counts[c2c[sx, sy, sz]] > 0:
                        srcs.append(int(c2c[sx, sy, sz]))
        for sc in sorted(srcs):
            near.append((starts[c], counts[c], starts[sc], counts[sc], c))
    prob = Problem(SRC_LAPLACE, npts, npts, X=P, Y=P, meta={"levels": L})
    return prob, np.asarray(far, dtype=np.int64).reshape(-1, 6), np.asarray(near, dtype=np.int64).reshape(-1, 5), L


def gaussian_blocks(nblk: int = 256, size: int = 1024, ell: float = 0.3, offset: float = 2.0, seed: int = 0):
    """nblk independent (targets, sources) pairs of point clouds in separated unit
    cubes; returns lists of (m,3) and (n,3) arrays."""
    g = rng(seed)
    Xs, Ys = [], []
    for _ in range(nblk):
        X = g.random((size, 3))
        Y = g.random((size, 3))
        Y[:, 0] += offset
        Xs.append(X)
        Ys.append(Y)
    return np.stack(Xs), np.stack(Ys), ell


def rhs(n: int, nrhs: int, seed: int, dtype=np.float64) -> np.ndarray:
    return rng(seed).standard_normal((n, nrhs)).astype(dtype)


def block_initial_rows(blocks: np.ndarray, kmax: int, seed: int) -> np.ndarray:
    """Per-block I0 (block-local): the first min(kmax, nrows, ncols) entries of a
    seeded permutation of the block's rows; unused slots are 0."""
    g = rng(seed)
    out = np.zeros((len(blocks), kmax), dtype=np.int32)
    for b, (r0, nr, c0, nc) in enumerate(np.asarray(blocks)):
        kb = int(min(kmax, nr, nc))
        out[b, :kb] = g.permutation(int(nr))[:kb]
    return out


def block_sample_positions(blocks: np.ndarray, q: int, s: int, seed: int):
    """Per-block residual sample rows (nb x q) and columns (nb x s), block-local,
    uniform without replacement when the block is large enough."""
    g = rng(seed)
    Q = np.zeros((len(blocks), q), dtype=np.int32)
    S = np.zeros((len(blocks), s), dtype=np.int32)
    for b, (r0, nr, c0, nc) in enumerate(np.asarray(blocks)):
        Q[b] = g.choice(int(nr), size=q, replace=q > nr)
        S[b] = g.choice(int(nc), size=s, replace=s > nc)
    return Q, S


def dense_blocks(n: int = 1500, sizes=(1, 7, 40, 64, 65, 300, 900), seed: int = 0):
    """Random rectangular blocks of an n x n matrix, sizes drawn from `sizes`."""
    g = rng(seed)
    out = []
    for nr in sizes:
        for nc in sizes:
            r0 = int(g.integers(0, n - nr + 1)); c0 = int(g.integers(0, n - nc + 1))
            out.append((r0, nr, c0, nc))
    return np.asarray(out, dtype=np.int64)

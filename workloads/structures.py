"""Seeded generators of block-sparse matrices (numpy only, host side).

A matrix is returned as a :class:`BlockMatrix`: the dimension ``n``, the leaf
size ``b`` and the list of stored leaves ``(brow[i], bcol[i], vals[i])`` in
row-major (I, J) leaf order, each leaf a row-major ``b x b`` float64 block.
Leaf values are always drawn in that order, ``b*b`` values per leaf, from
``numpy.random.default_rng(seed)`` (PCG64), so every consumer sees identical
inputs for a given seed.

Seeds: matrix A of workload ``c`` uses ``SEED_A + c``, matrix B ``SEED_B + c``,
the target T ``SEED_T + c`` and the lattice jitter ``SEED_GEOM + c``; product
``i`` of the batched workload adds ``10 * i``.

Nothing here multiplies matrices: these are inputs only.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_A = 1000
SEED_B = 2000
SEED_T = 3000
SEED_GEOM = 4000


@dataclass
class BlockMatrix:
    """A block-sparse matrix given as a list of dense leaves."""

    n: int
    b: int
    brow: np.ndarray  # int32 [nblk]
    bcol: np.ndarray  # int32 [nblk]
    vals: np.ndarray  # float64 [nblk, b, b], row-major inside each leaf

    @property
    def nblocks(self) -> int:
        return int(self.brow.shape[0])

    @property
    def grid(self) -> int:
        return self.n // self.b

    def to_dense(self) -> np.ndarray:
        """Dense ``n x n`` float64 copy (small sizes only)."""
        out = np.zeros((self.n, self.n), dtype=np.float64)
        b = self.b
        for i in range(self.nblocks):
            r, c = int(self.brow[i]), int(self.bcol[i])
            out[r * b:(r + 1) * b, c * b:(c + 1) * b] = self.vals[i]
        return out


def _rowmajor(rows: np.ndarray, cols: np.ndarray, grid: int):
    """Sort a leaf list into row-major (I, J) order."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.argsort(rows * grid + cols, kind="stable")
    return rows[order].astype(np.int32), cols[order].astype(np.int32)


def _uniform_leaves(rng, nblk: int, b: int) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, size=(nblk, b, b))


# --------------------------------------------------------------------------
# Banded leaves (the paper's "Banded" sequence, Section 3, at leaf level)
# --------------------------------------------------------------------------

def banded(n: int, b: int, half_width: int, seed: int) -> BlockMatrix:
    """Leaf (I, J) stored iff |I - J| <= half_width; entries U[-1, 1]."""
    if n % b:
        raise ValueError("n must be a multiple of b")
    g = n // b
    rows, cols = [], []
    for i in range(g):
        lo, hi = max(0, i - half_width), min(g - 1, i + half_width)
        rows.extend([i] * (hi - lo + 1))
        cols.extend(range(lo, hi + 1))
    brow, bcol = _rowmajor(np.array(rows), np.array(cols), g)
    rng = np.random.default_rng(seed)
    vals = _uniform_leaves(rng, brow.shape[0], b)
    return BlockMatrix(n, b, brow, bcol, vals)


# --------------------------------------------------------------------------
# Element-level structures of the paper's weak-scaling sequences (Section 3,
# Table 1): a band of half-width w united with dense diagonal blocks
# --------------------------------------------------------------------------

def structure_column_counts(n: int, half_width: int, blocks=()) -> np.ndarray:
    """Nonzeros of every column of the n x n element structure
    {(r, c): |r - c| <= w} united with the dense blocks [p, p+s)^2 of
    ``blocks`` (pairs (p, s), pairwise disjoint).  The structure is
    symmetric, so row counts are the same."""
    k = np.arange(n, dtype=np.int64)
    w = half_width
    c = np.minimum(k, w) + np.minimum(n - 1 - k, w) + 1
    for p, sz in blocks:
        kk = k[p:p + sz]
        lo = np.minimum(p, np.maximum(kk - w, 0))
        hi = np.maximum(p + sz - 1, np.minimum(kk + w, n - 1))
        c[p:p + sz] = hi - lo + 1
    return c


def structure_flops(n: int, half_width: int, blocks=()) -> int:
    """Element-level flops of the structure times itself,
    2 sum_k nnz(A[:, k]) nnz(A[k, :]) (the paper's Tflop rows)."""
    c = structure_column_counts(n, half_width, blocks)
    sq = c * c  # <= n^2 each; partial sums of 65536 stay below 2^63 for n < 1.1e7
    return 2 * sum(int(x) for x in np.add.reduceat(sq, np.arange(0, n, 65536)))


def _closest_size(flops_of, target: int, hi: int) -> int:
    lo = 1
    while lo < hi:  # smallest size reaching the target
        m = (lo + hi) // 2
        if flops_of(m) >= target:
            hi = m
        else:
            lo = m + 1
    best = lo
    if lo > 1 and abs(flops_of(lo - 1) - target) <= abs(flops_of(lo) - target):
        best = lo - 1
    return best


def growing_block_size(n: int, half_width: int) -> int:
    """Size of the dense top-left block for which the band plus the block
    needs twice the banded flops (the size with the closest flop count)."""
    target = 2 * structure_flops(n, half_width)
    return _closest_size(lambda s: structure_flops(n, half_width, [(0, s)]), target, n)


def random_blocks_layout(n: int, half_width: int, count: int, seed: int):
    """``count`` equal dense diagonal blocks at random positions, one in each
    of ``count`` equal slots of the diagonal, at least ``half_width`` from
    the slot's ends (so blocks neither overlap nor reach the matrix edge, and
    the flop count does not depend on the positions).  Their size is the one
    with the flop count closest to twice the banded flops.  Returns the list
    of (p, s)."""
    slot = n // count
    target = 2 * structure_flops(n, half_width)

    def flops_of(sz):
        return structure_flops(n, half_width,
                               [(i * slot + half_width, sz) for i in range(count)])

    sz = _closest_size(flops_of, target, slot - 2 * half_width)
    if slot - sz - 2 * half_width < 0:
        raise ValueError("blocks do not fit their slots")
    rng = np.random.default_rng(seed)
    offs = rng.integers(0, slot - sz - 2 * half_width + 1, size=count)
    return [(int(i * slot + half_width + o), int(sz)) for i, o in enumerate(offs)]


def band_with_blocks(n: int, b: int, half_width: int, blocks, seed: int) -> BlockMatrix:
    """The element structure of ``structure_column_counts`` stored in b x b
    leaves: the dimension is n rounded up to a multiple of b (rows and
    columns >= n are empty), a leaf is stored iff it holds a structural
    entry, structural entries are U[-1, 1] and the rest of a stored leaf is
    zero.  Leaf values are drawn for all stored leaves (row-major leaf order)
    and then masked."""
    npad = -(-n // b) * b
    g = npad // b
    gn = -(-n // b)  # leaf rows that hold matrix rows
    wl = (half_width + b - 1) // b
    keys = set()
    for i in range(gn):
        for j in range(max(0, i - wl), min(gn - 1, i + wl) + 1):
            keys.add(i * g + j)
    for p, sz in blocks:
        lo, hi = p // b, (p + sz - 1) // b
        for i in range(lo, hi + 1):
            keys.update(i * g + np.arange(lo, hi + 1))
    key = np.array(sorted(int(k) for k in keys), dtype=np.int64)
    brow, bcol = (key // g).astype(np.int32), (key % g).astype(np.int32)
    rng = np.random.default_rng(seed)
    vals = _uniform_leaves(rng, key.shape[0], b)
    e = np.arange(b, dtype=np.int64)
    chunk = 4096
    for s0 in range(0, key.shape[0], chunk):
        r = brow[s0:s0 + chunk].astype(np.int64)[:, None, None] * b + e[None, :, None]
        c = bcol[s0:s0 + chunk].astype(np.int64)[:, None, None] * b + e[None, None, :]
        m = np.abs(r - c) <= half_width
        for p, sz in blocks:
            m |= (r >= p) & (r < p + sz) & (c >= p) & (c < p + sz)
        m &= (r < n) & (c < n)
        vals[s0:s0 + chunk] *= m
    return BlockMatrix(npad, b, brow, bcol, vals)


def table1_structure(kind: str, n: int, b: int, half_width: int = 3000, count: int = 1,
                     seed: int = SEED_A + 6) -> tuple:
    """One matrix of the paper's weak-scaling sequences: kind 'banded',
    'growing_block' or 'random_blocks' (``count`` blocks).  Returns
    (BlockMatrix, blocks, element-level flops of its square)."""
    if kind == "banded":
        blocks = []
    elif kind == "growing_block":
        blocks = [(0, growing_block_size(n, half_width))]
    elif kind == "random_blocks":
        blocks = random_blocks_layout(n, half_width, count, seed + 7)
    else:
        raise ValueError(kind)
    m = band_with_blocks(n, b, half_width, blocks, seed)
    return m, blocks, structure_flops(n, half_width, blocks)


# --------------------------------------------------------------------------
# 3D locality: jittered cubic lattice ordered along a Morton curve
# --------------------------------------------------------------------------

def lattice_dims_for(npts: int):
    """Power-of-two lattice box (nx, ny, nz) with nx <= ny <= nz holding
    at least ``npts`` points: 8192 -> 16x16x32, 16384 -> 16x32x32,
    32768 -> 32x32x32, 65536 -> 32x32x64."""
    p = max(0, math.ceil(math.log2(max(1, npts))))
    e = [p // 3] * 3
    for k in range(p % 3):
        e[2 - k] += 1
    return tuple(1 << v for v in e)


def _morton3(x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    key = np.zeros(x.shape, dtype=np.int64)
    for bit in range(21):
        key |= ((x >> bit) & 1) << (3 * bit)
        key |= ((y >> bit) & 1) << (3 * bit + 1)
        key |= ((z >> bit) & 1) << (3 * bit + 2)
    return key


def lattice_points(npts: int, seed: int, jitter: float = 0.25) -> np.ndarray:
    """First ``npts`` points, in Morton order, of a power-of-two cubic lattice
    box with spacing 1, each coordinate jittered by i.i.d. U[-jitter, jitter].

    The jitter is drawn for the whole box (box-point count x 3, Morton order)
    before the first ``npts`` points are kept.  Returns float64 [npts, 3]."""
    nx, ny, nz = lattice_dims_for(npts)
    gx, gy, gz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    gx, gy, gz = gx.ravel(), gy.ravel(), gz.ravel()
    order = np.argsort(_morton3(gx, gy, gz), kind="stable")
    pts = np.stack([gx[order], gy[order], gz[order]], axis=1).astype(np.float64)
    rng = np.random.default_rng(seed)
    pts += rng.uniform(-jitter, jitter, size=pts.shape)
    return pts[:npts]


def locality_pattern(points: np.ndarray, b: int, cutoff: float):
    """Leaves (I, J), row-major, whose point groups (``b`` consecutive points
    each) come closer than ``cutoff``: min_{p in I, q in J} |x_p - x_q| < cutoff."""
    npts = points.shape[0]
    if npts % b:
        raise ValueError("point count must be a multiple of b")
    g = npts // b
    grp = points.reshape(g, b, 3)
    lo, hi = grp.min(axis=1), grp.max(axis=1)
    # bounding-box distance is a lower bound of the point-set distance
    gap = np.maximum(0.0, np.maximum(lo[:, None, :] - hi[None, :, :],
                                     lo[None, :, :] - hi[:, None, :]))
    cand = (gap ** 2).sum(axis=2) < cutoff * cutoff
    ci, cj = np.nonzero(np.triu(cand))
    keep = np.zeros(ci.shape[0], dtype=bool)
    c2 = cutoff * cutoff
    step = max(1, (1 << 22) // (b * b))
    for s in range(0, ci.shape[0], step):
        pi, pj = grp[ci[s:s + step]], grp[cj[s:s + step]]
        c = pi.mean(axis=1, keepdims=True)
        pi, pj = pi - c, pj - c
        d2 = ((pi * pi).sum(axis=2)[:, :, None] + (pj * pj).sum(axis=2)[:, None, :]
              - 2.0 * np.matmul(pi, pj.transpose(0, 2, 1)))
        keep[s:s + step] = d2.reshape(d2.shape[0], -1).min(axis=1) < c2
    ci, cj = ci[keep], cj[keep]
    rows = np.concatenate([ci, cj[ci != cj]])
    cols = np.concatenate([cj, ci[ci != cj]])
    return _rowmajor(rows, cols, g)


def locality_decay(points: np.ndarray, b: int, pattern) -> np.ndarray:
    """exp(-0.5 |x_p - x_q|) for every element (p, q) of the given leaves,
    float64 [nblk, b, b] (distances from the expansion |u|^2 + |v|^2 - 2 u.v
    of the points centred on the row group's mean)."""
    brow, bcol = pattern
    npts = points.shape[0]
    grp = points.reshape(npts // b, b, 3)
    out = np.empty((brow.shape[0], b, b), dtype=np.float64)
    step = max(1, (1 << 22) // (b * b))
    for s in range(0, brow.shape[0], step):
        pi, pj = grp[brow[s:s + step]], grp[bcol[s:s + step]]
        c = pi.mean(axis=1, keepdims=True)
        pi, pj = pi - c, pj - c
        d2 = ((pi * pi).sum(axis=2)[:, :, None] + (pj * pj).sum(axis=2)[:, None, :]
              - 2.0 * np.matmul(pi, pj.transpose(0, 2, 1)))
        np.maximum(d2, 0.0, out=d2)
        np.sqrt(d2, out=d2)
        d2 *= -0.5
        np.exp(d2, out=out[s:s + step])
    return out


def locality_matrix(points: np.ndarray, b: int, cutoff: float,
                    seed: int, pattern=None, decay=None) -> BlockMatrix:
    """3D-locality matrix: entry (p, q) of a stored leaf is
    exp(-0.5 |x_p - x_q|) * U[-1, 1] (``decay`` may be precomputed with
    locality_decay on the same pattern and shared between matrices)."""
    npts = points.shape[0]
    if pattern is None:
        pattern = locality_pattern(points, b, cutoff)
    brow, bcol = pattern
    rng = np.random.default_rng(seed)
    vals = _uniform_leaves(rng, brow.shape[0], b)
    if decay is None:
        decay = locality_decay(points, b, pattern)
    vals *= decay
    _ = npts
    return BlockMatrix(points.shape[0], b, brow, bcol, vals)


# --------------------------------------------------------------------------
# Random leaves
# --------------------------------------------------------------------------

def random_blocks(n: int, b: int, p: float, seed: int,
                  dist: str = "normal") -> BlockMatrix:
    """Each leaf stored independently with probability ``p`` (one U[0,1) draw
    per leaf of the grid, row-major, before the values); entries N(0, 1)
    (``dist='normal'``) or U[-1, 1] (``dist='uniform'``)."""
    g = n // b
    rng = np.random.default_rng(seed)
    present = rng.random((g, g)) < p
    rows, cols = np.nonzero(present)
    brow, bcol = rows.astype(np.int32), cols.astype(np.int32)
    if dist == "normal":
        vals = rng.standard_normal(size=(brow.shape[0], b, b))
    else:
        vals = _uniform_leaves(rng, brow.shape[0], b)
    return BlockMatrix(n, b, brow, bcol, vals)


def dense_line_pair(n: int, b: int, half_width: int, seed: int):
    """(A, B): A banded (|I - J| <= half_width leaves) plus a full first leaf
    row, B banded plus a full first leaf column, U[-1, 1] entries.  Leaf
    (0, 0) of A*B then sums n/b leaf pairs while every other leaf sums a
    handful: a product with one very long pair segment."""
    g = n // b
    out = []
    for t, sd in ((0, seed), (1, seed + 1)):
        keys = set()
        for i in range(g):
            for j in range(max(0, i - half_width), min(g - 1, i + half_width) + 1):
                keys.add(i * g + j)
        for j in range(g):
            keys.add(j if t == 0 else j * g)
        key = np.array(sorted(keys), dtype=np.int64)
        rng = np.random.default_rng(sd)
        vals = _uniform_leaves(rng, key.shape[0], b)
        out.append(BlockMatrix(n, b, (key // g).astype(np.int32), (key % g).astype(np.int32),
                               vals))
    return out[0], out[1]


def values_on_pattern(n: int, b: int, brow, bcol, seed: int) -> BlockMatrix:
    """N(0, 1) entries on every element of the given leaves (row-major order
    of the leaves is imposed first)."""
    g = n // b
    brow, bcol = _rowmajor(np.asarray(brow), np.asarray(bcol), g)
    rng = np.random.default_rng(seed)
    vals = rng.standard_normal(size=(brow.shape[0], b, b))
    return BlockMatrix(n, b, brow, bcol, vals)


def reblock(m: BlockMatrix, b_new: int) -> BlockMatrix:
    """The same element-level matrix stored with leaf size ``b_new`` (a
    multiple of ``m.b``), zero-filling the parts of a new leaf that no old
    leaf covers."""
    if b_new % m.b or m.n % b_new:
        raise ValueError("b_new must be a multiple of b and divide n")
    f = b_new // m.b
    g_new = m.n // b_new
    nr = m.brow.astype(np.int64) // f
    nc = m.bcol.astype(np.int64) // f
    key = nr * g_new + nc
    uniq, inv = np.unique(key, return_inverse=True)
    vals = np.zeros((uniq.shape[0], b_new, b_new), dtype=np.float64)
    sr = (m.brow.astype(np.int64) % f) * m.b
    sc = (m.bcol.astype(np.int64) % f) * m.b
    for i in range(m.nblocks):
        vals[inv[i], sr[i]:sr[i] + m.b, sc[i]:sc[i] + m.b] = m.vals[i]
    return BlockMatrix(m.n, b_new, (uniq // g_new).astype(np.int32),
                       (uniq % g_new).astype(np.int32), vals)


def symmetrize(m: BlockMatrix) -> BlockMatrix:
    """(M + M^T) / 2 on the union of M's leaf pattern and its transpose, in
    row-major leaf order: a symmetric input for the symmetric square."""
    g = m.grid
    b = m.b
    key = m.brow.astype(np.int64) * g + m.bcol.astype(np.int64)
    tkey = m.bcol.astype(np.int64) * g + m.brow.astype(np.int64)
    allk = np.unique(np.concatenate([key, tkey]))
    vals = np.zeros((allk.shape[0], b, b), dtype=np.float64)
    vals[np.searchsorted(allk, key)] += 0.5 * m.vals
    vals[np.searchsorted(allk, tkey)] += 0.5 * np.transpose(m.vals, (0, 2, 1))
    return BlockMatrix(m.n, b, (allk // g).astype(np.int32), (allk % g).astype(np.int32), vals)


def gershgorin_bounds(m: BlockMatrix):
    """(lo, hi) enclosing every eigenvalue of the symmetric matrix m
    (Gershgorin discs: diagonal entry -+ the off-diagonal absolute row sum).
    Used to map a matrix's spectrum into [0, 1] before purification."""
    b = m.b
    absrow = np.zeros(m.n)
    diag = np.zeros(m.n)
    rows = (m.brow.astype(np.int64)[:, None] * b + np.arange(b)[None, :]).reshape(-1)
    np.add.at(absrow, rows, np.abs(m.vals).sum(axis=2).reshape(-1))
    on = m.brow == m.bcol
    if np.any(on):
        d = np.diagonal(m.vals[on], axis1=1, axis2=2)
        drows = (m.brow[on].astype(np.int64)[:, None] * b + np.arange(b)[None, :]).reshape(-1)
        diag[drows] = d.reshape(-1)
    radius = absrow - np.abs(diag)
    return float(np.min(diag - radius)), float(np.max(diag + radius))


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

def config1(n: int = 4096, b: int = 32, half_width: int = 4):
    """Banded x banded: leaf (I, J) present iff |I - J| <= 4, U[-1, 1]."""
    return (banded(n, b, half_width, SEED_A + 1),
            banded(n, b, half_width, SEED_B + 1))


def config2(n: int = 65536, b: int = 64, cutoff: float = 6.0):
    """3D locality x 3D locality on one shared jittered lattice."""
    pts = lattice_points(n, SEED_GEOM + 2)
    pat = locality_pattern(pts, b, cutoff)
    dec = locality_decay(pts, b, pat)
    return (locality_matrix(pts, b, cutoff, SEED_A + 2, pattern=pat, decay=dec),
            locality_matrix(pts, b, cutoff, SEED_B + 2, pattern=pat, decay=dec))


def config2_symmetric(n: int = 65536, b: int = 64, cutoff: float = 6.0):
    """The symmetric 3D-locality matrix (A + A^T) / 2 of workload 2, the
    input of the symmetric square C = A^2."""
    return symmetrize(config2(n, b, cutoff)[0])


def config3(n: int = 32768, b: int = 32, p: float = 0.01):
    """Random leaves with probability p, N(0, 1) entries."""
    return (random_blocks(n, b, p, SEED_A + 3),
            random_blocks(n, b, p, SEED_B + 3))


def config5(n: int = 32768, b: int = 64, half_width: int = 8,
            cutoff: float = 6.0):
    """Banded (+-8 leaves) A times 3D-locality B; T is drawn later on the
    product's pattern with :func:`values_on_pattern` and seed SEED_T + 5."""
    a = banded(n, b, half_width, SEED_A + 5)
    pts = lattice_points(n, SEED_GEOM + 5)
    bm = locality_matrix(pts, b, cutoff, SEED_B + 5)
    return a, bm


def batched_products(count: int = 64, n_min: int = 2048, n_max: int = 32768,
                     seed: int = SEED_GEOM + 4, scale: float = 1.0):
    """The batched workload: ``count`` independent products C_i = A_i B_i.

    N_i = floor(exp(U[ln n_min, ln n_max])) rounded down to a multiple of 64
    (optionally multiplied by ``scale`` first, for reduced-size tests).
    Structure cycles with i mod 3: banded |I-J| <= 4 on 32-point leaves;
    3D locality with cutoff 6 on 64-point groups (first N_i points of a
    Morton-ordered power-of-two lattice box); random leaves with p = 0.02 on
    32-point leaves.  Every matrix is returned at leaf size 32 (3D leaves are
    split into their four 32x32 quarters), i.e. as the element-level matrix
    that a leaf-size choice then re-blocks.

    Returns a list of (kind, A, B)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ln = rng.uniform(math.log(n_min), math.log(n_max))
        n = int(math.floor(math.exp(ln) * scale)) // 64 * 64
        n = max(n, 64)
        kind = ("banded", "locality", "random")[i % 3]
        sa, sb = SEED_A + 4 + 10 * i, SEED_B + 4 + 10 * i
        if kind == "banded":
            a, bm = banded(n, 32, 4, sa), banded(n, 32, 4, sb)
        elif kind == "locality":
            pts = lattice_points(n, SEED_GEOM + 4 + 10 * i)
            pat = locality_pattern(pts, 64, 6.0)
            dec = locality_decay(pts, 64, pat)
            a = _split_leaves(locality_matrix(pts, 64, 6.0, sa, pattern=pat, decay=dec), 32)
            bm = _split_leaves(locality_matrix(pts, 64, 6.0, sb, pattern=pat, decay=dec), 32)
        else:
            a = random_blocks(n, 32, 0.02, sa)
            bm = random_blocks(n, 32, 0.02, sb)
        out.append((kind, a, bm))
    return out


def _split_leaves(m: BlockMatrix, b_new: int) -> BlockMatrix:
    """The same matrix with every leaf cut into (b/b_new)^2 smaller leaves
    (row-major leaf order)."""
    f = m.b // b_new
    nblk = m.nblocks * f * f
    brow = (m.brow.astype(np.int64)[:, None, None] * f
            + np.arange(f)[None, :, None]).repeat(f, axis=2).reshape(nblk)
    bcol = (m.bcol.astype(np.int64)[:, None, None] * f
            + np.arange(f)[None, None, :]).repeat(f, axis=1).reshape(nblk)
    vals = m.vals.reshape(m.nblocks, f, b_new, f, b_new).transpose(0, 1, 3, 2, 4)
    vals = vals.reshape(nblk, b_new, b_new)
    g = m.n // b_new
    order = np.argsort(brow * g + bcol, kind="stable")
    return BlockMatrix(m.n, b_new, brow[order].astype(np.int32),
                       bcol[order].astype(np.int32), np.ascontiguousarray(vals[order]))

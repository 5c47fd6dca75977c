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

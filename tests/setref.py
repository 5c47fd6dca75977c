"""Set-based and closed-form references used by the tests.

These are textbook definitions written with Python sets and numpy, kept apart
from both the CPU oracle and the GPU library.
"""

from __future__ import annotations

from collections import Counter, defaultdict

import numpy as np


def pattern_set(brow, bcol) -> set:
    return set(zip(np.asarray(brow).tolist(), np.asarray(bcol).tolist()))


def boolean_product(pa: set, pb: set) -> set:
    """{(I, J) : exists K with (I, K) in pa and (K, J) in pb}."""
    by_row = defaultdict(list)
    for k, j in pb:
        by_row[k].append(j)
    out = set()
    for i, k in pa:
        for j in by_row.get(k, ()):
            out.add((i, j))
    return out


def pair_count(pa: set, pb: set) -> int:
    """sum_K colcount_A(K) * rowcount_B(K): the number of (A-leaf, B-leaf)
    pairs that meet on a shared inner index K."""
    ca = Counter(k for _, k in pa)
    rb = Counter(k for k, _ in pb)
    return sum(ca[k] * rb.get(k, 0) for k in ca)


def upper_pair_count(pa: set, pb: set) -> int:
    """The pairs (I, K) x (K, J) with I <= J: for every K, the rows I of
    column K of pa against the columns J of row K of pb."""
    rows, cols = defaultdict(list), defaultdict(list)
    for i, k in pa:
        rows[k].append(i)
    for k, j in pb:
        cols[k].append(j)
    total = 0
    for k, ri in rows.items():
        cj = np.sort(np.asarray(cols.get(k, []), dtype=np.int64))
        if cj.size:
            total += int(np.sum(cj.size - np.searchsorted(cj, np.asarray(ri), side="left")))
    return total


def pairs_per_c_leaf(pa: set, pb: set) -> dict:
    """{(I, J): sorted list of K} for every contributing triple (I, K, J)."""
    by_row = defaultdict(list)
    for k, j in pb:
        by_row[k].append(j)
    out = defaultdict(list)
    for i, k in pa:
        for j in by_row.get(k, ()):
            out[(i, j)].append(k)
    return {c: sorted(ks) for c, ks in out.items()}


def product_pattern_counts(a_row, a_col, b_row, b_col, grid: int):
    """The boolean block product with multiplicities, as a sparse matrix
    product of the 0/1 leaf patterns (scipy CSR x CSR): arrays (I, J, count)
    of every C leaf, count = the number of K with A(I, K) and B(K, J)
    stored, in row-major (I, J) order.  For patterns too large for the set
    versions above."""
    from scipy import sparse
    ones = lambda r, c: sparse.csr_matrix(
        (np.ones(len(r), dtype=np.int64), (np.asarray(r, np.int64), np.asarray(c, np.int64))),
        shape=(grid, grid))
    p = (ones(a_row, a_col) @ ones(b_row, b_col)).tocoo()
    order = np.lexsort((p.col, p.row))
    return (p.row[order].astype(np.int64), p.col[order].astype(np.int64),
            p.data[order].astype(np.int64))


def banded_column_counts(n: int, half_width: int) -> np.ndarray:
    """Nonzeros of each column of an n x n banded matrix, |i - j| <= w."""
    k = np.arange(n, dtype=np.int64)
    return np.minimum(k, half_width) + np.minimum(n - 1 - k, half_width) + 1


def growing_block_column_counts(n: int, half_width: int, s: int) -> np.ndarray:
    """Column counts of the band united with a dense s x s top-left block."""
    k = np.arange(n, dtype=np.int64)
    c = banded_column_counts(n, half_width)
    c[:s] = np.maximum(s, np.minimum(k[:s] + half_width + 1, n))
    return c


def symmetric_square_flops(colcount: np.ndarray) -> int:
    """Flops of A*A for symmetric A: 2 sum_k nnz(A[:, k]) * nnz(A[k, :])."""
    return int(2 * (colcount.astype(np.int64) ** 2).sum())


def rel_fro(x: np.ndarray, ref: np.ndarray) -> float:
    den = float(np.linalg.norm(ref))
    num = float(np.linalg.norm(x - ref))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / den

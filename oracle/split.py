"""CPU oracle of the split-precision product (numpy, exact integer arithmetic).

TEST INFRASTRUCTURE ONLY: used by the tests and nothing else.

The split form (an Ozaki-style error-free splitting; Ozaki, Ogita, Oishi and
Rump, Numer. Algorithms 59, 2012) writes each FP64 operand as a short sum of
narrow slices so that slice products are exact in a low-precision unit:

1. Row scaling of A: e_r is the exponent with max_k |a_rk| in [2^(e_r-1),
   2^e_r) (frexp); column scaling of B: f_c likewise over column c.
2. Fixed point with s*w bits: A_int = trunc(a_rk * 2^(s*w - e_r)), so
   |A_int| < 2^(s*w); the same for B with f_c.
3. Signed base-2^w digits, most significant first:
   A_int = sum_{i=1..s} d_i 2^(w(s-i)),  |d_i| <= 2^w - 1,
   every digit carrying the sign of A_int.  With w <= 8 each digit is exactly
   representable in bfloat16 (8 significant bits).
4. C_rc ~= 2^(e_r + f_c - 2sw) sum_{(i,j) in S} 2^(w(2s-i-j)) sum_k d_i,rk g_j,kc
   over a chosen set S of slice pairs (usually i + j <= s + 1: the terms
   with larger i + j are below the truncation error).

Everything here is exact (Python integers) except the final conversion of
each result to FP64.  It is meant for small matrices.
"""

from __future__ import annotations

import numpy as np


def row_exponents(x: np.ndarray, axis: int) -> np.ndarray:
    """Per-row (axis=1) or per-column (axis=0) exponent e with
    max |x| in [2^(e-1), 2^e); 0 for an all-zero line."""
    m = np.max(np.abs(x), axis=axis)
    _, e = np.frexp(m)
    return np.where(m > 0, e, 0).astype(np.int64)


def fixed_point(x: np.ndarray, exps: np.ndarray, axis: int, s: int, w: int) -> np.ndarray:
    """trunc(x * 2^(s*w - e)) as exact integers (object array)."""
    shape = [1, 1]
    shape[1 - axis] = -1
    e = exps.reshape(shape)
    scaled = np.ldexp(x, (s * w - e).astype(np.int64))  # exact: a power-of-two scaling
    t = np.trunc(scaled)
    out = np.empty(x.shape, dtype=object)
    for idx, v in np.ndenumerate(t):
        out[idx] = int(v)
    return out


def digits(xi: np.ndarray, s: int, w: int) -> list:
    """Signed base-2^w digits d_1 (most significant) .. d_s of integers."""
    base = 1 << w
    out = []
    mags = np.vectorize(lambda v: abs(v), otypes=[object])(xi)
    signs = np.vectorize(lambda v: -1 if v < 0 else 1, otypes=[object])(xi)
    for i in range(1, s + 1):
        sh = w * (s - i)
        d = np.vectorize(lambda m: (m >> sh) % base, otypes=[object])(mags)
        out.append((d * signs).astype(np.int64))
    return out


def slice_pairs(s: int, extra: bool = False) -> list:
    """Slice pairs (i, j), 1-based, with i + j <= s + 1."""
    return [(i, j) for i in range(1, s + 1) for j in range(1, s + 1) if i + j <= s + 1]


def split_product(a: np.ndarray, b: np.ndarray, s: int, w: int, pairs=None,
                  sa: int | None = None):
    """Dense emulation of the split product of dense a (m x k) and b (k x n).
    ``sa`` digits are taken for A (default s; digit i keeps weight 2^(-w i)
    whatever the count), s for B.  Each S_ij = sum_k d_i g_j is an exact int64
    matrix product (|S_ij| <= k (2^w - 1)^2 < 2^63); the weighted sum over
    pairs and the final scaling are exact Python integers, rounded once.
    Returns (C_split as float64, e_row, f_col)."""
    if pairs is None:
        pairs = slice_pairs(s)
    sa = s if sa is None else sa
    e = row_exponents(a, axis=1)
    f = row_exponents(b, axis=0)
    da = digits(fixed_point(a, e, 1, sa, w), sa, w)
    db = digits(fixed_point(b, f, 0, s, w), s, w)
    m, n = a.shape[0], b.shape[1]
    top = max(i + j for i, j in pairs)
    acc = np.zeros((m, n), dtype=object)
    acc[:] = 0
    for i, j in pairs:
        sij = (da[i - 1] @ db[j - 1]).astype(object)
        acc = acc + sij * (1 << (w * (top - i - j)))
    out = np.empty((m, n), dtype=np.float64)
    for r in range(m):
        for c in range(n):
            out[r, c] = _to_double(acc[r, c], int(e[r]) + int(f[c]) - w * top)
    return out, e, f


def _to_double(v: int, exp2: int) -> float:
    """v * 2^exp2 rounded once to the nearest double."""
    if v == 0:
        return 0.0
    from fractions import Fraction
    q = Fraction(v) * (Fraction(2) ** exp2)
    return float(q)  # Fraction -> float rounds to nearest (ties to even)


def error_bound(a: np.ndarray, b: np.ndarray, s: int, w: int, kdim=None) -> np.ndarray:
    """Elementwise a-priori bound on |C_split - A B| for split_product with
    the pairs i + j <= s + 1:
       |C - C~|_rc <= 2^(e_r + f_c) * K * (s + 3) * 2^(-s*w)
    with K the inner dimension (truncation of each operand contributes
    < 2^(-s*w) relative to its line maximum < 2^e; each dropped slice pair
    i + j = s + 1 + q contributes at most K 2^(-w(s - 1 + q)) (1 - 2^-w)^2
    relative, and summing over q and over the at most s pairs per q stays
    below (s + 1) K 2^(-s*w))."""
    e = row_exponents(a, axis=1).astype(np.float64)
    f = row_exponents(b, axis=0).astype(np.float64)
    K = a.shape[1] if kdim is None else kdim
    return np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64)) * K * (s + 3) * 2.0 ** (-s * w)

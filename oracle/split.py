"""CPU oracle of the split-precision product (numpy, exact integer arithmetic).

TEST INFRASTRUCTURE ONLY: used by the tests and nothing else.

The split form (an Ozaki-style error-free splitting; Ozaki, Ogita, Oishi and
Rump, Numer. Algorithms 59, 2012) writes each FP64 operand as a short sum of
narrow slices so that slice products are exact in a low-precision unit:

1. Row scaling of A: e_r is the exponent with max_k |a_rk| in [2^(e_r-1),
   2^e_r) (frexp); column scaling of B: f_c likewise over column c.
2. Fixed point with s*w bits: A_int = round(a_rk * 2^(s*w - 1 - e_r))
   (halves away from zero), so |A_int| <= 2^(s*w - 1); the same for B.
3. Balanced signed base-2^w digits, most significant first:
   A_int = sum_{i=1..s} d_i 2^(w(s-i)),  |d_i| <= 2^(w-1),
   so that a_rk ~= 2^(e_r + 1) sum_i d_i 2^(-w i).  With w <= 8 each digit
   is exactly representable in bfloat16, and a product of two digits is at
   most 2^(2w - 2) in magnitude.
4. C_rc ~= 2^(e_r + f_c + 2) sum_{(i,j) in S} 2^(-w(i+j)) sum_k d_i,rk g_j,kc
   over a chosen set S of slice pairs (usually i + j <= s + 1: the terms
   with larger i + j are below the rounding error).

Everything here is exact (Python integers) except the final conversion of
each result to FP64.  It is meant for small matrices.
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def row_exponents(x: np.ndarray, axis: int) -> np.ndarray:
    """Per-row (axis=1) or per-column (axis=0) exponent e with
    max |x| in [2^(e-1), 2^e); 0 for an all-zero line."""
    m = np.max(np.abs(x), axis=axis)
    _, e = np.frexp(m)
    return np.where(m > 0, e, 0).astype(np.int64)


def fixed_point(x: np.ndarray, exps: np.ndarray, axis: int, s: int, w: int) -> np.ndarray:
    """round(x * 2^(s*w - 1 - e)) (halves away from zero) as exact integers,
    e the line exponent; |result| <= 2^(s*w - 1) because |x| < 2^e."""
    shape = [1, 1]
    shape[1 - axis] = -1
    e = np.broadcast_to(exps.reshape(shape), x.shape)
    out = np.empty(x.shape, dtype=object)
    half = Fraction(1, 2)
    for idx, v in np.ndenumerate(x):
        q = Fraction(float(v)) * Fraction(2) ** (s * w - 1 - int(e[idx]))
        m = math.floor(abs(q) + half)
        out[idx] = -m if q < 0 else m
    return out


def digits(xi: np.ndarray, s: int, w: int) -> list:
    """Balanced base-2^w digits d_1 (most significant) .. d_s of integers
    with |x| <= 2^(s*w - 1): the digits of |x| are taken from the least
    significant one in [-(2^(w-1) - 1), 2^(w-1)], then the sign of x is
    applied, so every |d_i| <= 2^(w-1) (the most significant one absorbs the
    remainder and stays in that range)."""
    base = 1 << w
    lo = (base >> 1) - 1

    def split(v):
        m = abs(v)
        ds = []
        for _ in range(s):
            t = (m + lo) % base - lo
            ds.append(t)
            m = (m - t) >> w
        assert m == 0, "integer out of range for s balanced digits"
        sg = -1 if v < 0 else 1
        return [sg * t for t in reversed(ds)]

    per = np.empty(xi.shape + (s,), dtype=np.int64)
    for idx, v in np.ndenumerate(xi):
        per[idx] = split(int(v))
    return [per[..., i] for i in range(s)]


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
            # a = 2^(e+1) sum_i d_i 2^(-w i), likewise b: weight 2^(e+f+2)
            out[r, c] = _to_double(acc[r, c], int(e[r]) + int(f[c]) + 2 - w * top)
    return out, e, f


def _to_double(v: int, exp2: int) -> float:
    """v * 2^exp2 rounded once to the nearest double."""
    if v == 0:
        return 0.0
    q = Fraction(v) * (Fraction(2) ** exp2)
    return float(q)  # Fraction -> float rounds to nearest (ties to even)


def error_bound(a: np.ndarray, b: np.ndarray, s: int, w: int, kdim=None) -> np.ndarray:
    """Elementwise a-priori bound on |C_split - A B| for split_product with
    the pairs i + j <= s + 1:
       |C - C~|_rc <= 2^(e_r + f_c) * K * (s + 3) * 2^(-s*w)
    with K the inner dimension.  Per term a_rk b_kc, with a = 2^(e+1) (X + dx)
    and b = 2^(f+1) (Y + dy), |X|, |Y| <= 1/2 and |dx|, |dy| <= 2^(-s*w-1)
    (rounding): the representation error is below 2^(e+f+2) 2^(-s*w-1) (1 +
    2^(-s*w)) = 2^(e+f) 2 2^(-s*w) (1 + 2^(-s*w)), and each dropped slice
    pair i + j = s + 1 + q (at most s of them, j fixing i) is at most
    2^(e+f+2) 2^(2w-2) 2^(-w(s+1+q)) = 2^(e+f) 2^(-w(s-1+q)), which sums over
    q >= 1 to below 2^(e+f) s 2^(-s*w) / (1 - 2^-w); together below
    2^(e+f) (s + 3) 2^(-s*w) per term."""
    e = row_exponents(a, axis=1).astype(np.float64)
    f = row_exponents(b, axis=0).astype(np.float64)
    K = a.shape[1] if kdim is None else kdim
    return np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64)) * K * (s + 3) * 2.0 ** (-s * w)

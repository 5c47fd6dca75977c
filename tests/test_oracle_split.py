"""Pins of the split-precision oracle (oracle/split.py) against mathematics:
exact digit reconstruction, bfloat16-representable digits, exact products of
small-integer matrices, the a-priori error bound, and convergence to the
FP64 product as the number of slices grows."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import split as sp


def _rand(shape, seed, scale_rows=False):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=shape)
    if scale_rows:
        x *= np.exp2(rng.integers(-20, 20, size=(shape[0], 1)))
    return x


@pytest.mark.parametrize("s,w", [(6, 8), (7, 7), (4, 8), (8, 6)])
def test_digits_reconstruct_fixed_point(s, w):
    a = _rand((12, 20), 1, scale_rows=True)
    e = sp.row_exponents(a, axis=1)
    ai = sp.fixed_point(a, e, 1, s, w)
    d = sp.digits(ai, s, w)
    back = sum(d[i].astype(object) * (1 << (w * (s - 1 - i))) for i in range(s))
    assert np.all(back == ai)
    for di in d:
        assert np.all(np.abs(di) <= 1 << (w - 1))
    # rounding to nearest: |x 2^(sw - 1 - e) - A_int| <= 1/2, signs agree,
    # and |A_int| <= 2^(sw - 1)
    scaled = np.ldexp(a, (s * w - 1 - e)[:, None])
    diff = scaled - ai.astype(np.float64)
    assert np.all(np.abs(diff) <= 0.5 * (1 + 1e-15) + np.spacing(np.abs(scaled)))
    assert np.all((ai.astype(np.float64) == 0) | (np.sign(ai.astype(np.float64)) == np.sign(a)))
    assert all(abs(int(v)) <= 1 << (s * w - 1) for v in ai.ravel())


def test_balanced_digits_of_the_extremes():
    # the largest magnitude 2^(sw - 1) and values around digit boundaries
    s, w = 3, 8
    vals = np.array([1 << 23, -(1 << 23), 127, 128, 129, -127, -128, -129, 255, 256,
                     (1 << 23) - 1, -((1 << 23) - 1), 0], dtype=object)
    d = sp.digits(vals, s, w)
    for k, v in enumerate(vals):
        ds = [int(d[i][k]) for i in range(s)]
        assert sum(t << (w * (s - 1 - i)) for i, t in enumerate(ds)) == v
        assert all(abs(t) <= 128 for t in ds)
    with pytest.raises(AssertionError):
        sp.digits(np.array([(1 << 23) + (1 << 16)], dtype=object), s, w)


def test_digits_are_bfloat16_exact():
    torch = pytest.importorskip("torch")
    a = _rand((16, 16), 2)
    e = sp.row_exponents(a, axis=1)
    for di in sp.digits(sp.fixed_point(a, e, 1, 6, 8), 6, 8):
        t = torch.from_numpy(di.astype(np.float64))
        assert torch.equal(t.to(torch.bfloat16).to(torch.float64), t)


def test_row_exponent_brackets_the_row_max():
    a = _rand((10, 7), 3, scale_rows=True)
    e = sp.row_exponents(a, axis=1)
    m = np.abs(a).max(axis=1)
    assert np.all(m < np.ldexp(1.0, e)) and np.all(m >= np.ldexp(0.5, e))
    z = np.zeros((2, 3))
    assert np.all(sp.row_exponents(z, axis=1) == 0)


def test_small_integer_matrices_are_exact():
    rng = np.random.default_rng(4)
    a = rng.integers(-100, 101, size=(9, 11)).astype(np.float64)
    b = rng.integers(-100, 101, size=(11, 8)).astype(np.float64)
    c, _, _ = sp.split_product(a, b, s=2, w=8)
    assert np.array_equal(c, a @ b)


@pytest.mark.parametrize("s,w", [(3, 8), (4, 7), (5, 8), (6, 8), (7, 7)])
def test_error_within_bound(s, w):
    a = _rand((16, 24), 5, scale_rows=True)
    b = _rand((24, 12), 6)
    c, _, _ = sp.split_product(a, b, s, w)
    exact = a.astype(np.longdouble) @ b.astype(np.longdouble)
    err = np.abs(c - exact.astype(np.float64))
    bound = sp.error_bound(a, b, s, w) + 2 * np.spacing(np.abs(exact.astype(np.float64)))
    assert np.all(err <= bound)


def test_converges_to_fp64_product():
    a = _rand((20, 32), 7)
    b = _rand((32, 20), 8)
    ref = a @ b
    errs = []
    for s in (2, 3, 4, 5, 6):
        c, _, _ = sp.split_product(a, b, s, 8)
        errs.append(np.linalg.norm(c - ref) / np.linalg.norm(ref))
    assert all(errs[i + 1] < errs[i] / 16 for i in range(3))
    assert errs[-1] < 1e-13


def test_zero_rows_and_columns():
    a = _rand((6, 5), 9)
    b = _rand((5, 4), 10)
    a[2] = 0.0
    b[:, 1] = 0.0
    c, e, f = sp.split_product(a, b, 6, 8)
    assert np.all(c[2] == 0.0) and np.all(c[:, 1] == 0.0)
    assert e[2] == 0 and f[1] == 0

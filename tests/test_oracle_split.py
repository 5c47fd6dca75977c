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


# ------------------------------------------------------- planted mistakes --
# Each mutant replaces one step of the split oracle with a plausible mistake
# (on the CPU, by patching the module); the pins above must catch every one.

def _digits_unbalanced(xi, s, w):
    # plain base-2^w digits of |x| with the sign applied: up to 2^w - 1
    base = 1 << w
    per = np.empty(xi.shape + (s,), dtype=np.int64)
    for idx, v in np.ndenumerate(xi):
        m, ds = abs(int(v)), []
        for _ in range(s):
            ds.append(m % base)
            m >>= w
        sg = -1 if v < 0 else 1
        per[idx] = [sg * t for t in reversed(ds)]
    return [per[..., i] for i in range(s)]


def _digits_lost_sign(xi, s, w):
    return [np.abs(d) for d in _ORIG["digits"](xi, s, w)]


def _fixed_point_truncating(x, exps, axis, s, w):
    import math
    from fractions import Fraction
    shape = [1, 1]
    shape[1 - axis] = -1
    e = np.broadcast_to(exps.reshape(shape), x.shape)
    out = np.empty(x.shape, dtype=object)
    for idx, v in np.ndenumerate(x):
        q = Fraction(float(v)) * Fraction(2) ** (s * w - 1 - int(e[idx]))
        m = math.floor(abs(q))
        out[idx] = -m if q < 0 else m
    return out


def _row_exponents_high(x, axis):
    e = _ORIG["row_exponents"](x, axis)
    return np.where(np.max(np.abs(x), axis=axis) > 0, e + 1, e)


def _slice_pairs_short(s, extra=False):
    return [(i, j) for i in range(1, s + 1) for j in range(1, s + 1) if i + j <= s]


def _to_double_doubled(v, exp2):
    return _ORIG["_to_double"](v, exp2 + 1)


_ORIG = {name: getattr(sp, name) for name in
         ("digits", "fixed_point", "row_exponents", "slice_pairs", "_to_double")}
_MUTANTS = {
    "unbalanced_digits": ("digits", _digits_unbalanced),
    "lost_digit_sign": ("digits", _digits_lost_sign),
    "truncating_fixed_point": ("fixed_point", _fixed_point_truncating),
    "exponent_one_high": ("row_exponents", _row_exponents_high),
    "dropped_diagonal": ("slice_pairs", _slice_pairs_short),
    "doubled_scale": ("_to_double", _to_double_doubled),
}


def _split_pins_hold() -> bool:
    pins = (lambda: test_digits_reconstruct_fixed_point(6, 8),
            test_balanced_digits_of_the_extremes,
            test_row_exponent_brackets_the_row_max,
            test_small_integer_matrices_are_exact,
            lambda: test_error_within_bound(6, 8),
            test_converges_to_fp64_product,
            test_zero_rows_and_columns)
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            return False
    return True


def test_split_pins_hold_unmutated():
    assert _split_pins_hold()


@pytest.mark.parametrize("mutant", list(_MUTANTS))
def test_split_pins_catch_planted_mistakes(monkeypatch, mutant):
    name, fn = _MUTANTS[mutant]
    monkeypatch.setattr(sp, name, fn)
    assert not _split_pins_hold()

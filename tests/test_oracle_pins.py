"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or mathematics fixes:
a dense product computed independently, identity and zero products, the
boolean-product pattern computed with sets, the pair-count closed form and
the paper's Table 1, associativity, transposition and the gradient formula
(checked by exact finite differences).  The last test plants plausible
mistakes in copies of the oracle and shows that these pins catch each one.
"""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
import workloads as w
from tests import setref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _om(m, mutant=0):
    return oracle.OMatrix.from_block_matrix(m, mutant)


def _tiny_pair(n, b, p, seed):
    a = w.random_blocks(n, b, p, seed, dist="uniform")
    bm = w.random_blocks(n, b, p, seed + 1, dist="uniform")
    return a, bm


def _triple_loop(x, y):
    n = x.shape[0]
    out = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            s = 0.0
            for k in range(n):
                s += x[i, k] * y[k, j]
            out[i, j] = s
    return out


def _identity(n, b):
    g = n // b
    idx = np.arange(g, dtype=np.int32)
    vals = np.broadcast_to(np.eye(b), (g, b, b)).copy()
    return w.BlockMatrix(n, b, idx, idx.copy(), vals)


# ---------------------------------------------------------------- products --

@pytest.mark.parametrize("n,b,p,seed", [(24, 4, 0.4, 1), (32, 8, 0.5, 2),
                                        (20, 4, 0.3, 3), (12, 2, 0.6, 4)])
def test_matches_python_triple_loop(n, b, p, seed):
    a, bm = _tiny_pair(n, b, p, seed)
    c = _om(a) @ _om(bm)
    ref = _triple_loop(a.to_dense(), bm.to_dense())
    assert setref.rel_fro(c.to_dense(), ref) <= 1e-14


@pytest.mark.parametrize("n,b,p,seed", [(64, 8, 0.3, 5), (96, 8, 0.2, 6),
                                        (40, 8, 0.5, 7), (64, 1, 0.1, 8)])
def test_matches_dense_numpy(n, b, p, seed):
    a, bm = _tiny_pair(n, b, p, seed)
    c = _om(a) @ _om(bm)
    ref = a.to_dense() @ bm.to_dense()
    assert setref.rel_fro(c.to_dense(), ref) <= 1e-13


def test_identity_is_exact():
    a = w.banded(96, 8, 2, 11)
    eye = _identity(96, 8)
    left = _om(eye) @ _om(a)
    right = _om(a) @ _om(eye)
    assert np.array_equal(left.to_dense(), a.to_dense())
    assert np.array_equal(right.to_dense(), a.to_dense())
    assert left.pattern() == setref.pattern_set(a.brow, a.bcol)


def test_zero_operand_gives_nil():
    a = w.banded(64, 8, 1, 12)
    empty = w.BlockMatrix(64, 8, np.zeros(0, np.int32), np.zeros(0, np.int32),
                          np.zeros((0, 8, 8)))
    zeros = w.BlockMatrix(64, 8, a.brow.copy(), a.bcol.copy(),
                          np.zeros_like(a.vals))
    for z in (empty, zeros):
        c, npairs = _om(a).multiply(_om(z))
        assert c.nleaves() == 0 and npairs == 0
        c, npairs = _om(z).multiply(_om(a))
        assert c.nleaves() == 0 and npairs == 0


def test_all_zero_input_leaves_are_nil():
    a = w.banded(64, 8, 1, 13)
    a.vals[3] = 0.0
    m = _om(a)
    assert m.nleaves() == a.nblocks - 1
    assert (int(a.brow[3]), int(a.bcol[3])) not in m.pattern()


@pytest.mark.parametrize("n,b,p,seed", [(80, 8, 0.2, 21), (56, 8, 0.35, 22),
                                        (128, 4, 0.05, 23)])
def test_pattern_is_boolean_product(n, b, p, seed):
    a, bm = _tiny_pair(n, b, p, seed)
    c, npairs = _om(a).multiply(_om(bm))
    pa, pb = setref.pattern_set(a.brow, a.bcol), setref.pattern_set(bm.brow, bm.bcol)
    assert c.pattern() == setref.boolean_product(pa, pb)
    assert npairs == setref.pair_count(pa, pb)


def test_cancelling_leaf_stays_in_pattern():
    # A(0,0) B(0,0) + A(0,1) B(1,0) = I - I = 0 stays structurally present
    b = 4
    eye = np.eye(b)
    a = w.BlockMatrix(8, b, np.array([0, 0], np.int32), np.array([0, 1], np.int32),
                      np.stack([eye, -eye]))
    bm = w.BlockMatrix(8, b, np.array([0, 1], np.int32), np.array([0, 0], np.int32),
                       np.stack([eye, eye]))
    c = _om(a) @ _om(bm)
    assert c.pattern() == {(0, 0)}
    assert np.all(c.to_dense() == 0.0)


def test_config1_pair_count_and_pattern():
    a, bm = w.config1()
    c, npairs = _om(a).multiply(_om(bm))
    pa, pb = setref.pattern_set(a.brow, a.bcol), setref.pattern_set(bm.brow, bm.bcol)
    assert npairs == setref.pair_count(pa, pb) == 10068
    assert c.nleaves() == 2104
    assert c.pattern() == setref.boolean_product(pa, pb)


def test_element_level_banded_pair_count():
    # leaf size 1: the recursion's leaf products are the scalar multiplications
    n, hw = 200, 7
    a = w.banded(n, 1, hw, 31)
    _, npairs = _om(a).multiply(_om(a))
    cc = setref.banded_column_counts(n, hw)
    assert 2 * npairs == setref.symmetric_square_flops(cc)


def test_associativity():
    a, bm = _tiny_pair(64, 8, 0.3, 41)
    cm = w.random_blocks(64, 8, 0.3, 43, dist="uniform")
    A, B, C = _om(a), _om(bm), _om(cm)
    left = (A @ B) @ C
    right = A @ (B @ C)
    assert left.pattern() == right.pattern()
    assert setref.rel_fro(left.to_dense(), right.to_dense()) <= 1e-12


def test_leaf_product_matches_recursion():
    a, bm = w.config1(512, 32)
    A, B = _om(a), _om(bm)
    c = A @ B
    brow, bcol, vals = c.leaves()
    for idx in [0, 7, len(brow) // 2, len(brow) - 1]:
        v, present = oracle.leaf_product(A, B, int(brow[idx]), int(bcol[idx]))
        assert present
        assert setref.rel_fro(v, vals[idx]) <= 1e-14
    _, present = oracle.leaf_product(A, B, 0, 15)
    assert not present


def test_non_power_of_two_grid():
    for n, b in [(40, 8), (56, 8), (24, 8), (8, 8)]:
        a, bm = _tiny_pair(n, b, 0.6, n)
        c = _om(a) @ _om(bm)
        assert setref.rel_fro(c.to_dense(), a.to_dense() @ bm.to_dense()) <= 1e-14


def test_extract_is_morton_order():
    a = w.random_blocks(256, 8, 0.2, 51)
    brow, bcol, _ = _om(a).leaves()
    keys = oracle.morton_key(brow, bcol)
    assert np.all(np.diff(keys) > 0)
    assert len(brow) == a.nblocks


def test_rejects_bad_input():
    a = w.banded(64, 8, 1, 61)
    with pytest.raises(oracle.OracleError) as e:
        oracle.OMatrix.from_blocks(64, 8, np.r_[a.brow, a.brow[:1]],
                                   np.r_[a.bcol, a.bcol[:1]],
                                   np.concatenate([a.vals, a.vals[:1]]))
    assert e.value.code == -3
    with pytest.raises(oracle.OracleError) as e:
        oracle.OMatrix.from_blocks(64, 8, np.array([8], np.int32),
                                   np.array([0], np.int32), np.ones((1, 8, 8)))
    assert e.value.code == -1
    with pytest.raises(oracle.OracleError):
        oracle.OMatrix.from_blocks(60, 8, a.brow, a.bcol, a.vals)
    b16 = w.banded(64, 16, 1, 62)
    with pytest.raises(oracle.OracleError) as e:
        _om(a).multiply(_om(b16))
    assert e.value.code == -2


def test_transpose():
    a = w.random_blocks(48, 8, 0.4, 71, dist="uniform")
    t = _om(a).transpose()
    assert np.array_equal(t.to_dense(), a.to_dense().T)


# --------------------------------------------------------------- backward --

def test_backward_matches_dense_formula():
    a, bm = _tiny_pair(64, 8, 0.3, 81)
    A, B = _om(a), _om(bm)
    c = A @ B
    cb, cc, cv = c.leaves()
    tgt = w.values_on_pattern(64, 8, cb, cc, 83)
    T = _om(tgt)
    dcv = 2.0 * (c.to_dense() - T.to_dense())
    mask_c = (c.to_dense() != 0) | (T.to_dense() != 0)
    dc_blocks = w.BlockMatrix(64, 8, cb, cc,
                              np.stack([dcv[r * 8:(r + 1) * 8, q * 8:(q + 1) * 8]
                                        for r, q in zip(cb, cc)]))
    dA, dB = oracle.backward(A, B, _om(dc_blocks))
    ad, bd = a.to_dense(), bm.to_dense()
    mask_a = np.kron(_leaf_mask(a), np.ones((8, 8)))
    mask_b = np.kron(_leaf_mask(bm), np.ones((8, 8)))
    assert dA.pattern() == setref.pattern_set(a.brow, a.bcol)
    assert dB.pattern() == setref.pattern_set(bm.brow, bm.bcol)
    assert setref.rel_fro(dA.to_dense(), (dcv @ bd.T) * mask_a) <= 1e-13
    assert setref.rel_fro(dB.to_dense(), (ad.T @ dcv) * mask_b) <= 1e-13
    assert mask_c.any()


def _leaf_mask(m):
    g = m.n // m.b
    out = np.zeros((g, g))
    out[m.brow, m.bcol] = 1.0
    return out


def test_backward_finite_differences():
    # L(A, B) = ||A B - T||_F^2 is quadratic in every single entry, so a
    # central difference has no truncation error: only rounding remains.
    n, b = 32, 4
    a, bm = _tiny_pair(n, b, 0.5, 91)
    A, B = _om(a), _om(bm)
    c = A @ B
    cb, cc, _ = c.leaves()
    tgt = w.values_on_pattern(n, b, cb, cc, 93).to_dense()
    ad, bd = a.to_dense(), bm.to_dense()

    def loss(x, y):
        return float(((x @ y - tgt) ** 2).sum())

    dcv = 2.0 * (c.to_dense() - tgt)
    dc_m = w.BlockMatrix(n, b, cb, cc, np.stack(
        [dcv[r * b:(r + 1) * b, q * b:(q + 1) * b] for r, q in zip(cb, cc)]))
    dA, dB = oracle.backward(A, B, _om(dc_m))
    gA, gB = dA.to_dense(), dB.to_dense()
    rng = np.random.default_rng(95)
    h = 1e-3
    for which, grad, base in (("A", gA, ad), ("B", gB, bd)):
        m = a if which == "A" else bm
        for _ in range(24):
            leaf = rng.integers(m.nblocks)
            i = int(m.brow[leaf]) * b + int(rng.integers(b))
            j = int(m.bcol[leaf]) * b + int(rng.integers(b))
            xp, xm = base.copy(), base.copy()
            xp[i, j] += h
            xm[i, j] -= h
            if which == "A":
                fd = (loss(xp, bd) - loss(xm, bd)) / (2 * h)
            else:
                fd = (loss(ad, xp) - loss(ad, xm)) / (2 * h)
            assert abs(fd - grad[i, j]) <= 1e-8 * max(1.0, abs(fd))


# ----------------------------------------------------------- paper's Table 1 --

def _printed_close(x: float, printed: float) -> bool:
    """x agrees with a value printed to four significant digits."""
    exp = int(np.floor(np.log10(abs(printed))))
    return abs(x - printed) <= 0.5 * 10.0 ** (exp - 3) + 1e-12


def test_table1_flop_counts():
    g = json.load(open(os.path.join(GOLDEN, "table1_weak_scaling.json")))
    hw = g["banded_half_width"]
    for n, tf in zip(g["matrix_size"], g["banded_tflop"]):
        flops = setref.symmetric_square_flops(setref.banded_column_counts(n, hw))
        assert _printed_close(flops / 1e12, tf), (n, flops / 1e12, tf)
    for n, s, tf in zip(g["matrix_size"], g["growing_block_size"],
                        g["growing_block_tflop"]):
        cc = setref.growing_block_column_counts(n, hw, s)
        flops = setref.symmetric_square_flops(cc)
        assert _printed_close(flops / 1e12, tf), (n, s, flops / 1e12, tf)
        # the added block doubles the work (Section 3)
        base = setref.symmetric_square_flops(setref.banded_column_counts(n, hw))
        assert abs(flops / base - 2.0) < 2e-3


def test_largest_banded_bytes():
    g = json.load(open(os.path.join(GOLDEN, "table1_weak_scaling.json")))
    n = g["matrix_size"][-1]
    nnz = int(setref.banded_column_counts(n, g["banded_half_width"]).sum())
    gb = nnz * 8 / 1e9
    assert round(gb) == g["largest_banded_gigabytes_fp64"]
    # the text's "3.8 billion" nonzeros is 38.4 billion: 307 GB fixes it
    assert 3.8e10 < nnz < 3.9e10


# ------------------------------------------------------- planted mistakes --

def _pins_hold(mutant: int) -> bool:
    try:
        a, bm = _tiny_pair(32, 4, 0.5, 101)
        A = oracle.OMatrix.from_block_matrix(a, mutant)
        B = oracle.OMatrix.from_block_matrix(bm, mutant)
        c, npairs = A.multiply(B)
        if setref.rel_fro(c.to_dense(), a.to_dense() @ bm.to_dense()) > 1e-13:
            return False
        pa = setref.pattern_set(a.brow, a.bcol)
        pb = setref.pattern_set(bm.brow, bm.bcol)
        if c.pattern() != setref.boolean_product(pa, pb):
            return False
        if npairs != setref.pair_count(pa, pb):
            return False
        eye = _identity(32, 4)
        E = oracle.OMatrix.from_block_matrix(eye, mutant)
        if not np.array_equal((A @ E).to_dense(), a.to_dense()):
            return False
        return True
    except oracle.OracleError:
        return False


def test_pins_hold_for_oracle():
    assert _pins_hold(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4])
def test_pins_catch_planted_mistakes(mutant):
    # 1 drops a term of the quadrant sum, 2 transposes the left leaf operand,
    # 3 flips the sign of the added product, 4 takes B's quadrants transposed
    assert not _pins_hold(mutant)

"""GPU split-precision form (BF16 slices on tcgen05) against the oracles.

Two comparisons:
1. with the exact emulation of the same splitting (oracle/split.py, the same
   slice pairs as the kernel's MMA blocks): only the FP32 rounding of the two
   low-weight TMEM regions and the final rounding separate them;
2. with the FP64 product: within the a-priori bound of the splitting, and the
   relative Frobenius error is reported.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from oracle import split as sp
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu

S, W = 6, 8


def _kernel_pairs(b):
    """Slice pairs the kernel's MMA blocks compute: block (u, j) stacks A
    slices u.. along M and B slices j, j+1 along N."""
    if b == 64:
        blocks = [(1, 1), (1, 3), (3, 1), (1, 5), (3, 3), (5, 1)]
        parts, sa = 2, 6
    else:
        blocks = [(1, 1), (1, 3), (1, 5), (5, 1)]
        parts, sa = 4, 8
    return sorted({(u + p, j + q) for u, j in blocks for p in range(parts)
                   for q in range(2)}), sa


FEW = 4  # C leaves of at most this many leaf pairs go to the one-pair kernel


def _single_pairs():
    """Slice pairs of the kernel for C leaves of at most FEW leaf pairs
    (32-leaves): the slice pairs (i, j) with i + j <= 7, per leaf pair, summed
    exactly.  A keeps its 8 digits (only 1..6 meet a B digit)."""
    return sp.slice_pairs(S), 8


def _one_pair_mask(plan, n, b):
    """Dense mask of the C leaves of the one-pair kernel: those that sum at
    most FEW leaf pairs."""
    arr = plan.arrays()
    seg = np.diff(arr["cseg"].numpy())
    few = seg <= FEW
    out = np.zeros((n, n), dtype=bool)
    for r, c in zip(arr["crow"].numpy()[few], arr["ccol"].numpy()[few]):
        out[r * b:(r + 1) * b, c * b:(c + 1) * b] = True
    return out


def _emulate(lib, plan, ad, bd, b, n):
    """The exact emulation of the split product with, for every C leaf, the
    slice pairs of the kernel that computes it: at b = 32 the leaves of at
    most FEW leaf pairs (grouped by B leaf) and the others (the general
    kernel) differ.  Returns (emulation, e, f, mask of the one-pair kernel's
    leaves or None)."""
    pairs, sa = _kernel_pairs(b)
    emu, e, f = sp.split_product(ad, bd, S, W, pairs=pairs, sa=sa)
    if b != 32 or not lib.get_option(lib.OPT_SPLIT_SINGLE):
        return emu, e, f, None
    one = _one_pair_mask(plan, n, b)
    if one.any():
        p1, sa1 = _single_pairs()
        emu1, _, _ = sp.split_product(ad, bd, S, W, pairs=p1, sa=sa1)
        emu = np.where(one, emu1, emu)
    return emu, e, f, one


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


def _dense_on(M, n):
    br, bc, v = gu.host_leaves(M)
    out = np.zeros((n, n))
    b = M.b
    for i in range(len(br)):
        out[br[i] * b:(br[i] + 1) * b, bc[i] * b:(bc[i] + 1) * b] = v[i]
    return out


@pytest.mark.parametrize("b,n,p", [(64, 256, 0.6), (32, 256, 0.5), (64, 192, 1.0),
                                   (32, 96, 1.0)])
def test_split_matches_exact_emulation(lib, b, n, p):
    a = w.random_blocks(n, b, p, 11 + b, dist="uniform")
    bm = w.random_blocks(n, b, p, 12 + b, dist="normal")
    a.vals *= np.exp2(np.random.default_rng(5).integers(-12, 12, size=(a.nblocks, b, 1)))
    A, B = gu.upload(lib, a), gu.upload(lib, bm)
    plan = lib.cht_symbolic_multiply(A, B)
    C, bound = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    got = _dense_on(C, n)
    ad, bd = a.to_dense(), bm.to_dense()
    emu, e, f, one = _emulate(lib, plan, ad, bd, b, n)
    scale = np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64))
    mask = _dense_on(C, n) != 0
    # FP32 rounding in the two low TMEM regions (weight 2^-48 and 2^-56 of
    # 2^(e_r + f_c)): at most (steps) * 2^-23 * (partial sum <= 3 K 2^16),
    # steps <= 3 K / 16 per C leaf, so < 2^-54 K^2 relative, K = inner length
    tol = scale * float(n) ** 2 * 2.0 ** -54 + 2 * np.spacing(np.abs(emu))
    if one is not None:
        # one-pair leaves: every diagonal exact in FP32 and in the int64
        # assembly, so only the final rounding to double remains
        tol = np.where(one, 2 * np.spacing(np.abs(emu)), tol)
    diff = np.abs(got - emu)
    assert np.all(diff[mask] <= tol[mask]), float((diff / tol).max())
    ref = ad @ bd
    within = np.abs(got - ref) <= sp.error_bound(ad, bd, S, W) + 2 * np.spacing(np.abs(ref))
    assert np.all(within)
    assert 0 < bound < 1e-6


@pytest.mark.parametrize("b", [64, 32])
def test_split_wide_exponent_range(lib, b):
    # rows of A and columns of B scaled by 2^s, s in [-540, 500]: C spans
    # about 2^-1070 .. 2^988, with huge, tiny and subnormal results (the
    # conversion of the integer result falls back to ldexp below the normal
    # range)
    n = 256 if b == 64 else 128
    a = w.random_blocks(n, b, 0.7, 41 + b, dist="uniform")
    bm = w.random_blocks(n, b, 0.7, 42 + b, dist="uniform")
    rng = np.random.default_rng(43)
    sr, sc = rng.integers(-520, 481, size=n), rng.integers(-520, 481, size=n)
    sr[:4] = [-540, 500, 0, -1]
    sc[:4] = [-530, 480, -520, 3]
    for i in range(a.nblocks):
        r0 = int(a.brow[i]) * b
        a.vals[i] = np.ldexp(a.vals[i], sr[r0:r0 + b][:, None])
    for i in range(bm.nblocks):
        c0 = int(bm.bcol[i]) * b
        bm.vals[i] = np.ldexp(bm.vals[i], sc[c0:c0 + b][None, :])
    A, B = gu.upload(lib, a), gu.upload(lib, bm)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    got = _dense_on(C, n)
    emu, e, f, _ = _emulate(lib, plan, a.to_dense(), bm.to_dense(), b, n)
    assert np.all(np.isfinite(got))
    assert np.any((got != 0) & (np.abs(got) < np.finfo(np.float64).tiny))  # subnormals
    assert np.abs(got).max() > 2.0 ** 900
    scale = np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64))
    tol = scale * float(n) ** 2 * 2.0 ** -54 + 2 * np.spacing(np.abs(emu))
    diff = np.abs(got - emu)
    assert np.all(diff <= tol), float((diff / tol).max())


@pytest.mark.parametrize("name", ["banded_4096_b32", "locality_8192_b64", "random_4096_b32"])
def test_split_close_to_fp64(lib, name):
    if name == "banded_4096_b32":
        a, b = w.config1()
    elif name == "locality_8192_b64":
        a, b = w.config2(8192)
    else:
        a, b = (w.random_blocks(4096, 32, 0.03, 1003), w.random_blocks(4096, 32, 0.03, 2003))
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    Cs, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    Cd, _ = lib.cht_multiply(plan, A, B, sync=True)
    Co, _ = gu.oracle_product(a, b)
    gu.assert_same_pattern(Cs, Co)
    err = gu.assert_values_close(Cs, Co, 1e-12, leaf_tol=None)
    e64 = setref.rel_fro(Cs.values().cpu().numpy(), Cd.values().cpu().numpy())
    print(f"{name}: split vs oracle rel. Frobenius {err:.2e}, vs FP64 path {e64:.2e}")
    assert e64 <= 1e-12


def test_split_zero_rows_and_empty(lib):
    a = w.random_blocks(512, 64, 0.5, 21, dist="uniform")
    a.vals[:, 5, :] = 0.0  # an all-zero row inside every leaf
    b = w.random_blocks(512, 64, 0.5, 22, dist="uniform")
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    ref = a.to_dense() @ b.to_dense()
    got = C.to_dense().cpu().numpy()
    assert np.all(got[5::64] == 0.0)
    assert setref.rel_fro(got, ref) <= 1e-12
    empty = w.BlockMatrix(512, 64, np.zeros(0, np.int32), np.zeros(0, np.int32),
                          np.zeros((0, 64, 64)))
    E = gu.upload(lib, empty)
    plan = lib.cht_symbolic_multiply(A, E)
    C, _ = lib.cht_multiply(plan, A, E, mode=lib.CHT_SPLIT_BF16, sync=True)
    assert C.nblocks == 0


def test_split_long_segments(lib):
    # many pairs per C leaf: many exact windows per leaf (dense 12 x 12 grid)
    a = w.random_blocks(768, 64, 1.0, 31, dist="uniform")
    b = w.random_blocks(768, 64, 1.0, 32, dist="uniform")
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    ref = a.to_dense() @ b.to_dense()
    got = C.to_dense().cpu().numpy()
    bound = sp.error_bound(a.to_dense(), b.to_dense(), S, W)
    assert np.all(np.abs(got - ref) <= bound + 2 * np.spacing(np.abs(ref)))
    assert setref.rel_fro(got, ref) <= 1e-12


def test_split_timeout_path(lib):
    a, b = w.config1(1024, 32, 2)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    old = lib.get_option(lib.OPT_WAIT_BUDGET_NS)
    lib.set_option(lib.OPT_WAIT_BUDGET_NS, 0)
    try:
        with pytest.raises(lib.ChtError) as e:
            lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
        assert e.value.code == lib.CHT_ERR_TIMEOUT
    finally:
        lib.set_option(lib.OPT_WAIT_BUDGET_NS, old)
    lib.sync_status()
    C, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    Co, _ = gu.oracle_product(a, b)
    gu.assert_values_close(C, Co, 1e-12, leaf_tol=None)
    _ = oracle


@pytest.mark.parametrize("b,g", [(64, 1100), (64, 2100), (32, 4100)])
def test_split_long_segments_are_cut_into_pieces(lib, b, g):
    # leaf (0, 0) of A*B sums g leaf pairs, more than one unit of the split
    # kernel sums (1016 at b = 64, 4000 at b = 32): it is computed in pieces
    a, bm = w.dense_line_pair(g * b, b, 1, 91)
    A, B = gu.upload(lib, a), gu.upload(lib, bm)
    plan = lib.cht_symbolic_multiply(A, B)
    OC, npairs = gu.oracle_product(a, bm)
    assert plan.npairs == npairs
    Cs, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    gu.assert_same_pattern(Cs, OC)
    gu.assert_values_close(Cs, OC, 1e-11, leaf_tol=None)
    _, _, ov = OC.leaves()
    assert setref.rel_fro(Cs.values()[0].cpu().numpy(), ov[0]) <= 1e-11


def test_full_size_random_sampled(lib):
    # the random-leaf workload at its full size (N = 32768, 32x32 leaves,
    # p = 0.01): pattern and pair counts from the set definitions, sampled C
    # leaves of both forms against the oracle's single-leaf product
    a, b = w.config3()
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    pa, pb = setref.pattern_set(a.brow, a.bcol), setref.pattern_set(b.brow, b.bcol)
    assert plan.npairs == setref.pair_count(pa, pb)
    assert plan.nnzb_C == len(setref.boolean_product(pa, pb))
    Cd, _ = lib.cht_multiply(plan, A, B, sync=True)
    Cs, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    arr = plan.arrays()
    crow, ccol = arr["crow"].numpy(), arr["ccol"].numpy()
    seglen = np.diff(arr["cseg"].numpy())
    OA, OB = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    vd, vs = Cd.values(), Cs.values()
    rng = np.random.default_rng(11)
    picks = list(rng.choice(crow.shape[0], 12, replace=False)) + [int(np.argmax(seglen))]
    for c in picks:
        ref, present = oracle.leaf_product(OA, OB, int(crow[c]), int(ccol[c]))
        assert present
        assert setref.rel_fro(vd[c].cpu().numpy(), ref) <= 1e-13
        assert setref.rel_fro(vs[c].cpu().numpy(), ref) <= 1e-11


def _one_pair_case(scaled: bool):
    """32-leaves, n = 256 (8 x 8 leaf grid): random leaves, plus a full leaf
    column 3 of A and B leaves (3, 1), (3, 5), (3, 6) alone in their
    columns, so that C leaves (I, 1), (I, 5), (I, 6) sum exactly one pair for
    every I: runs of 8 one-pair leaves per B leaf (two full groups of 4),
    next to leaves of one, two and more pairs elsewhere."""
    n, b, g = 256, 32, 8
    rng = np.random.default_rng(65 + int(scaled))
    pa = {(i, j) for i in range(g) for j in range(g) if rng.random() < 0.3} | \
        {(i, 3) for i in range(g)}
    pb = {(i, j) for i in range(g) for j in range(g)
          if rng.random() < 0.3 and j not in (1, 5, 6)} | {(3, 1), (3, 5), (3, 6)}

    def build(keys, dist):
        keys = sorted(keys)
        vals = (rng.standard_normal((len(keys), b, b)) if dist == "normal"
                else rng.uniform(-1, 1, (len(keys), b, b)))
        return w.BlockMatrix(n, b, np.array([k[0] for k in keys], np.int32),
                             np.array([k[1] for k in keys], np.int32), vals)

    a, bm = build(pa, "normal"), build(pb, "uniform")
    if scaled:  # rows of A and columns of B over a wide exponent range
        sr, sc = rng.integers(-60, 61, size=n), rng.integers(-60, 61, size=n)
        for i in range(a.nblocks):
            r0 = int(a.brow[i]) * b
            a.vals[i] = np.ldexp(a.vals[i], sr[r0:r0 + b][:, None])
        for i in range(bm.nblocks):
            c0 = int(bm.bcol[i]) * b
            bm.vals[i] = np.ldexp(bm.vals[i], sc[c0:c0 + b][None, :])
    return a, bm


@pytest.mark.parametrize("scaled", [False, True])
def test_split_one_pair_leaves(lib, scaled):
    # The leaf pairs of C leaves that sum at most FEW of them go to the kernel
    # that groups them by B leaf (up to 4 per MMA; a leaf of several pairs
    # has its exact integer results summed afterwards), the other C leaves
    # to the general kernel.  Each against the exact emulation of its own
    # slice pairs, the one-pair kernel's leaves to within the final
    # rounding; then the same product with the grouping switched off
    # (general kernel only) against its own pairs.
    n, b = 256, 32
    a, bm = _one_pair_case(scaled)
    A, B = gu.upload(lib, a), gu.upload(lib, bm)
    plan = lib.cht_symbolic_multiply(A, B)
    seg = np.diff(plan.arrays()["cseg"].numpy())
    assert (seg == 1).sum() >= 24 and ((seg >= 2) & (seg <= FEW)).sum() > 0
    ad, bd = a.to_dense(), bm.to_dense()
    mask = _dense_on(lib.cht_multiply(plan, A, B, sync=True)[0], n) != 0
    for single in (1, 0):
        lib.set_option(lib.OPT_SPLIT_SINGLE, single)
        try:
            C, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
            emu, e, f, one = _emulate(lib, plan, ad, bd, b, n)
        finally:
            lib.set_option(lib.OPT_SPLIT_SINGLE, 1)
        assert (one is not None) == bool(single)
        got = _dense_on(C, n)
        scale = np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64))
        tol = scale * float(n) ** 2 * 2.0 ** -54 + 2 * np.spacing(np.abs(emu))
        if one is not None:
            # exact up to the final rounding: the emulation's own result
            tol = np.where(one, 2 * np.spacing(np.abs(emu)), tol)
        diff = np.abs(got - emu)
        assert np.all(diff[mask] <= tol[mask]), (single, float((diff / tol).max()))
        assert np.all(got[~mask] == 0)
        ref = ad @ bd
        assert np.all(np.abs(got - ref) <= sp.error_bound(ad, bd, S, W)
                      + 2 * np.spacing(np.abs(ref)))
    lib.sync_status()


def test_split_pair_count_boundary(lib):
    """C leaves of 1 .. 5 leaf pairs (banded +-2 times banded +-2 on an 8 x 8
    leaf grid of 32-leaves): those of at most FEW pairs go to the one-pair
    kernel (the several-pair ones as one unit per pair, their exact integers
    summed and rounded once), those of FEW + 1 to the general kernel; each
    against the exact emulation of its own slice pairs."""
    n, b = 256, 32
    a, bm = w.banded(n, b, 2, 7071), w.banded(n, b, 2, 7072)
    A, B = gu.upload(lib, a), gu.upload(lib, bm)
    plan = lib.cht_symbolic_multiply(A, B)
    seg = np.diff(plan.arrays()["cseg"].numpy())
    assert set(seg.tolist()) == {1, 2, 3, 4, 5}
    C, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    ad, bd = a.to_dense(), bm.to_dense()
    emu, e, f, one = _emulate(lib, plan, ad, bd, b, n)
    assert one is not None and one.any() and not one.all()
    got = _dense_on(C, n)
    scale = np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64))
    tol = scale * float(n) ** 2 * 2.0 ** -54 + 2 * np.spacing(np.abs(emu))
    tol = np.where(one, 2 * np.spacing(np.abs(emu)), tol)
    mask = _dense_on(lib.cht_multiply(plan, A, B, sync=True)[0], n) != 0
    assert np.all(np.abs(got - emu)[mask] <= tol[mask])
    assert np.all(np.abs(got - ad @ bd) <= sp.error_bound(ad, bd, S, W)
                  + 2 * np.spacing(np.abs(ad @ bd)))
    lib.sync_status()

"""Pins of the weak-scaling structures (paper, Section 3 and Table 1): the
block-size rule reproduces every printed growing-block size, the
element-level flop counts reproduce the printed Tflop rows, the random
blocks double the banded flops wherever they sit, and the leaf-level
generator stores exactly the structure it describes."""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_weak_scaling.json")


@pytest.fixture(scope="module")
def table1():
    with open(GOLDEN) as f:
        return json.load(f)


def _tflop4(x):
    return float(f"{x / 1e12:.4g}")


def test_growing_block_sizes_reproduce_table1(table1):
    hw = table1["banded_half_width"]
    sizes = [w.growing_block_size(n, hw) for n in table1["matrix_size"]]
    assert sizes == table1["growing_block_size"]


def test_flop_rows_reproduce_table1(table1):
    hw = table1["banded_half_width"]
    for i, n in enumerate(table1["matrix_size"]):
        assert _tflop4(w.structure_flops(n, hw)) == table1["banded_tflop"][i]
        s = table1["growing_block_size"][i]
        assert _tflop4(w.structure_flops(n, hw, [(0, s)])) == table1["growing_block_tflop"][i]


def test_random_blocks_double_the_banded_flops(table1):
    hw = table1["banded_half_width"]
    for i, n in enumerate(table1["matrix_size"][:4]):
        count = table1["random_blocks_count"][i]
        lay1 = w.random_blocks_layout(n, hw, count, 1)
        lay2 = w.random_blocks_layout(n, hw, count, 2)
        assert len(lay1) == count and lay1 != lay2
        f1 = w.structure_flops(n, hw, lay1)
        assert f1 == w.structure_flops(n, hw, lay2)  # position independent
        # twice the banded flops to within one step of the block size, and
        # the printed Tflop (given to 4 digits) to within 1e-3
        fb = w.structure_flops(n, hw)
        assert abs(f1 - 2 * fb) <= 2e-4 * fb
        tf = table1["random_blocks_tflop"][i]
        assert abs(f1 / 1e12 - tf) <= 1e-3 * tf
        # disjoint, away from each other and from the edges by >= hw
        ends = sorted((p, p + s) for p, s in lay1)
        assert ends[0][0] >= hw and ends[-1][1] <= n - hw
        assert all(b0 - a1 >= 2 * hw for (_, a1), (b0, _) in zip(ends, ends[1:]))
        # the printed sizes come from positions the paper does not give;
        # ours stay within 1% of them
        s = lay1[0][1]
        assert abs(s - table1["random_blocks_size"][i]) <= 0.01 * s


@pytest.mark.parametrize("kind,count", [("banded", 1), ("growing_block", 1),
                                        ("random_blocks", 2)])
def test_leaf_generator_stores_the_structure(kind, count):
    n, b, hw = 1000, 32, 40  # n not a multiple of b: padded to 1024
    m, blocks, flops = w.table1_structure(kind, n, b, hw, count)
    assert m.n == 1024
    d = m.to_dense()
    r, c = np.indices((m.n, m.n))
    want = (np.abs(r - c) <= hw) & (r < n) & (c < n)
    for p, s in blocks:
        want |= (r >= p) & (r < p + s) & (c >= p) & (c < p + s)
    assert np.array_equal(d != 0, want)
    cc = want.sum(axis=0)[:n]
    assert np.array_equal(cc, w.structure_column_counts(n, hw, blocks))
    assert flops == 2 * int((cc.astype(np.int64) ** 2).sum())
    leaves = {(int(i), int(j)) for i, j in zip(*np.nonzero(
        want.reshape(m.n // b, b, m.n // b, b).any(axis=(1, 3))))}
    assert set(zip(m.brow.tolist(), m.bcol.tolist())) == leaves
    if kind == "growing_block":
        assert blocks == [(0, w.growing_block_size(n, hw))]

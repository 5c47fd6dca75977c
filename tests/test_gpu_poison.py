"""Every C leaf is written by the numeric phase: C is poisoned with NaN before
a second multiply into it, and the result equals the first bit for bit (FP64
and split forms; 32- and 64-leaves; a C leaf the split kernel computes in
pieces)."""

from __future__ import annotations

import pytest

import workloads as w
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

CASES = {
    "banded_4096_b32": lambda: w.config1(),
    # mostly one leaf pair per C leaf: the split form groups them by B leaf
    "random_8192_b32": lambda: (w.random_blocks(8192, 32, 0.02, 71),
                                w.random_blocks(8192, 32, 0.02, 72)),
    "locality_8192_b64": lambda: w.config2(8192),
    # leaf (0, 0) sums 1100 pairs: the split kernel cuts it into pieces
    "line_pair_70400_b64": lambda: w.dense_line_pair(1100 * 64, 64, 1, 91),
}


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_every_c_leaf_is_written(lib, name, mode):
    import torch
    a, b = CASES[name]()
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    m = lib.CHT_FP64 if mode == "fp64" else lib.CHT_SPLIT_BF16
    C, _ = lib.cht_multiply(plan, A, B, mode=m, sync=True)
    ref = C.values().clone()
    assert bool(torch.isfinite(ref).all())
    C.values().fill_(float("nan"))
    lib.cht_multiply(plan, A, B, mode=m, out=C, sync=True)
    assert torch.equal(C.values(), ref)

"""GPU products of the paper's weak-scaling structures (Section 3, Table 1):
band plus dense diagonal blocks, stored element-exactly in zero-padded
leaves.  Scaled-down cases against the oracle (pattern and pairs bit-exact,
values within the FP64 and split tolerances); the paper's first size,
N = 100000 with a 15716-wide top-left block, on sampled leaves."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


@pytest.mark.parametrize("kind,count,b", [("banded", 1, 32), ("growing_block", 1, 32),
                                          ("random_blocks", 3, 32), ("growing_block", 1, 64)])
def test_table1_structures_match_oracle(lib, kind, count, b):
    a, _, _ = w.table1_structure(kind, 4000, b, 120, count)
    A = gu.upload(lib, a)
    plan = lib.cht_symbolic_multiply(A, A)
    gu.check_plan_pairs(plan, a, a)
    OA = oracle.OMatrix.from_block_matrix(a)
    OC, npairs = OA.multiply(OA)
    assert plan.npairs == npairs
    C, _ = lib.cht_multiply(plan, A, A, sync=True)
    gu.assert_same_pattern(C, OC)
    gu.assert_values_close(C, OC, 1e-13)
    Cs, _ = lib.cht_multiply(plan, A, A, mode=lib.CHT_SPLIT_BF16, sync=True)
    gu.assert_values_close(Cs, OC, 1e-11, leaf_tol=None)


def test_paper_size_growing_block_sampled(lib):
    scipy_sparse = pytest.importorskip("scipy.sparse")
    a, blocks, eflops = w.table1_structure("growing_block", 100000, 64)
    assert blocks == [(0, 15716)] and f"{eflops / 1e12:.4g}" == "14.04"
    A = gu.upload(lib, a)
    plan = lib.cht_symbolic_multiply(A, A)
    pa = setref.pattern_set(a.brow, a.bcol)
    assert plan.npairs == setref.pair_count(pa, pa)
    g = a.grid
    P = scipy_sparse.csr_matrix((np.ones(a.nblocks), (a.brow, a.bcol)), shape=(g, g))
    assert plan.nnzb_C == (P @ P).nnz
    C, _ = lib.cht_multiply(plan, A, A, sync=True)
    arr = plan.arrays()
    crow, ccol = arr["crow"].numpy(), arr["ccol"].numpy()
    seglen = np.diff(arr["cseg"].numpy())
    OA = oracle.OMatrix.from_block_matrix(a)
    vals = C.values()
    rng = np.random.default_rng(9)
    picks = list(rng.choice(crow.shape[0], 10, replace=False)) + [int(np.argmax(seglen)), 0,
                                                                 crow.shape[0] - 1]
    for c in picks:
        ref, present = oracle.leaf_product(OA, OA, int(crow[c]), int(ccol[c]))
        assert present
        assert setref.rel_fro(vals[c].cpu().numpy(), ref) <= 1e-13

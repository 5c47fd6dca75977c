"""Helpers shared by the GPU tests: upload inputs, run the oracle, compare."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import setref


def cht():
    """The GPU library, or skip when no GPU is present."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_11762_gb300 as lib
    lib.load()
    return lib


def upload(lib, m):
    return lib.from_block_matrix(m)


def host_leaves(M):
    brow, bcol = M.coords()
    return (brow.cpu().numpy(), bcol.cpu().numpy(), M.values().cpu().numpy())


def oracle_product(a, b):
    A = oracle.OMatrix.from_block_matrix(a)
    B = oracle.OMatrix.from_block_matrix(b)
    C, npairs = A.multiply(B)
    return C, npairs


def assert_same_pattern(M, omat):
    gr, gc, _ = host_leaves(M)
    orow, ocol, _ = omat.leaves(values=False)
    assert np.array_equal(gr, orow) and np.array_equal(gc, ocol)


def assert_values_close(M, omat, tol=1e-13):
    _, _, gv = host_leaves(M)
    _, _, ov = omat.leaves()
    assert gv.shape == ov.shape
    err = setref.rel_fro(gv, ov)
    assert err <= tol, f"relative Frobenius error {err:.3e} > {tol:.1e}"
    return err


def check_plan_pairs(plan, a, b):
    """Pair segments of the plan equal the set-based triple lists, with K
    ascending inside every C leaf, bit for bit."""
    arr = plan.arrays()
    A_r, A_c = _morton_coords(a)
    B_r, B_c = _morton_coords(b)
    cseg = arr["cseg"].numpy()
    pa = arr["pair_a"].numpy()
    pb = arr["pair_b"].numpy()
    crow = arr["crow"].numpy()
    ccol = arr["ccol"].numpy()
    ref = setref.pairs_per_c_leaf(setref.pattern_set(a.brow, a.bcol),
                                  setref.pattern_set(b.brow, b.bcol))
    assert len(ref) == crow.shape[0]
    for c in range(crow.shape[0]):
        I, J = int(crow[c]), int(ccol[c])
        seg = slice(int(cseg[c]), int(cseg[c + 1]))
        ks_a = A_c[pa[seg]]
        ks_b = B_r[pb[seg]]
        assert np.array_equal(ks_a, ks_b)
        assert np.all(A_r[pa[seg]] == I) and np.all(B_c[pb[seg]] == J)
        assert ks_a.tolist() == ref[(I, J)]
    order = arr["order"].numpy()
    assert np.array_equal(np.sort(order), np.arange(crow.shape[0]))
    return arr


def _morton_coords(m):
    """Leaf coordinates of m in Morton order (the library's storage order),
    dropping all-zero leaves as the library does."""
    keep = np.any(m.vals.reshape(m.nblocks, -1) != 0, axis=1)
    r, c = m.brow[keep], m.bcol[keep]
    order = np.argsort(oracle.morton_key(r, c), kind="stable")
    return r[order], c[order]

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


_SAME = object()


def assert_values_close(M, omat, tol=1e-13, leaf_tol=_SAME):
    """Whole-matrix relative Frobenius error <= tol and, unless leaf_tol is
    None, the largest per-leaf relative Frobenius error <= leaf_tol (default:
    tol).  A leaf whose reference is exactly zero is measured against the
    root-mean-square leaf norm instead, so that a small wrong leaf cannot hide
    under the norm of the whole matrix.

    Callers pass leaf_tol=None for the split form, whose error is relative to
    the row and column maxima of the operands (the splitting scales whole
    lines), not to each leaf, and for truncated purification iterates, whose
    smallest kept leaves carry the cancellation of 3X^2 - 2X^3."""
    _, _, gv = host_leaves(M)
    _, _, ov = omat.leaves()
    assert gv.shape == ov.shape
    err = setref.rel_fro(gv, ov)
    assert err <= tol, f"relative Frobenius error {err:.3e} > {tol:.1e}"
    if leaf_tol is _SAME:
        leaf_tol = tol
    if leaf_tol is not None and ov.shape[0] > 0:
        worst, leaf = max_leaf_rel_err(gv, ov)
        assert worst <= leaf_tol, (f"leaf {leaf}: relative Frobenius error {worst:.3e} > "
                                   f"{leaf_tol:.1e}")
    return err


def max_leaf_rel_err(gv, ov):
    """(largest per-leaf relative Frobenius error, its leaf index)."""
    n = ov.shape[0]
    num = np.linalg.norm((gv - ov).reshape(n, -1), axis=1)
    den = np.linalg.norm(ov.reshape(n, -1), axis=1)
    rms = float(np.sqrt(np.mean(den * den)))
    den = np.where(den > 0, den, rms if rms > 0 else 1.0)
    rel = num / den
    i = int(np.argmax(rel))
    return float(rel[i]), i


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

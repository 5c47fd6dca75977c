"""GPU symmetric square C = A^2 (symmetric A): the upper-triangle plan
against the oracle's upper-triangle product (pattern and pair counts bit
exact, values within the FP64 and split tolerances), the mirrored full
matrix against the oracle's full product, and the edge cases."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13
SPLIT_TOL = 1e-11


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


def _case(name):
    if name == "locality":
        return w.config2_symmetric(8192)
    if name == "banded":
        return w.symmetrize(w.banded(4096, 32, 4, 71))
    return w.symmetrize(w.random_blocks(2048, 32, 0.05, 72))


@pytest.mark.parametrize("name", ["locality", "banded", "random"])
def test_symsquare_matches_oracle(lib, name):
    a = _case(name)
    A = gu.upload(lib, a)
    plan = lib.cht_symbolic_multiply_symsquare(A)
    OA = oracle.OMatrix.from_block_matrix(a)
    OU, npairs = OA.multiply_upper(OA)
    assert plan.npairs == npairs
    arr = plan.arrays()
    assert np.all(arr["crow"].numpy() <= arr["ccol"].numpy())
    U, _ = lib.cht_multiply(plan, A, A, sync=True)
    gu.assert_same_pattern(U, OU)
    gu.assert_values_close(U, OU, FP64_TOL)
    Us, _ = lib.cht_multiply(plan, A, A, mode=lib.CHT_SPLIT_BF16, sync=True)
    gu.assert_values_close(Us, OU, SPLIT_TOL, leaf_tol=None)
    # the mirrored upper triangle is the full product
    full = lib.cht_mat_mirror_upper(U)
    OC, _ = OA.multiply(OA)
    gu.assert_same_pattern(full, OC)
    gu.assert_values_close(full, OC, FP64_TOL)


def test_symsquare_pairs_are_the_upper_segments_of_the_full_plan(lib):
    a = _case("banded")
    A = gu.upload(lib, a)
    ps = lib.cht_symbolic_multiply_symsquare(A)
    pf = lib.cht_symbolic_multiply(A, A)
    xs, xf = ps.arrays(), pf.arrays()
    up = xf["crow"].numpy() <= xf["ccol"].numpy()
    assert np.array_equal(xs["crow"].numpy(), xf["crow"].numpy()[up])
    assert np.array_equal(xs["ccol"].numpy(), xf["ccol"].numpy()[up])
    segf = np.diff(xf["cseg"].numpy())[up]
    assert np.array_equal(np.diff(xs["cseg"].numpy()), segf)


def test_mirror_rejects_lower_leaves_and_handles_empty(lib):
    a = w.random_blocks(512, 32, 0.3, 73)
    assert np.any(a.brow > a.bcol)
    with pytest.raises(lib.ChtError):
        lib.cht_mat_mirror_upper(gu.upload(lib, a))
    e = w.BlockMatrix(512, 32, np.zeros(0, np.int32), np.zeros(0, np.int32),
                      np.zeros((0, 32, 32)))
    E = gu.upload(lib, e)
    plan = lib.cht_symbolic_multiply_symsquare(E)
    assert plan.npairs == 0
    U, _ = lib.cht_multiply(plan, E, E, sync=True)
    assert lib.cht_mat_mirror_upper(U).nblocks == 0


def test_mirror_transposes_off_diagonal_leaves(lib):
    # an upper-triangle matrix: its off-diagonal leaves come back transposed
    # below the diagonal, its diagonal leaves keep their upper triangles
    a = w.random_blocks(256, 32, 0.5, 74)
    up = a.brow <= a.bcol
    u = w.BlockMatrix(a.n, a.b, a.brow[up], a.bcol[up], a.vals[up])
    full = lib.cht_mat_mirror_upper(gu.upload(lib, u))
    ndiag = int(np.sum(u.brow == u.bcol))
    assert full.nblocks == 2 * u.nblocks - ndiag
    d = u.to_dense()
    # the element-level upper triangle of u, mirrored (diagonal leaves too)
    assert np.array_equal(full.to_dense().cpu().numpy(), np.triu(d) + np.triu(d, 1).T)


def test_full_size_symsquare_sampled(lib):
    # N = 65536, 64x64 leaves: pattern and pair counts exact, sampled upper
    # leaves against the oracle's single-leaf product
    a = w.config2_symmetric(65536)
    A = gu.upload(lib, a)
    plan = lib.cht_symbolic_multiply_symsquare(A)
    pa = setref.pattern_set(a.brow, a.bcol)
    assert plan.npairs == setref.upper_pair_count(pa, pa)
    U, _ = lib.cht_multiply(plan, A, A, sync=True)
    arr = plan.arrays()
    crow, ccol = arr["crow"].numpy(), arr["ccol"].numpy()
    full = setref.boolean_product(pa, pa)
    assert set(zip(crow.tolist(), ccol.tolist())) == {c for c in full if c[0] <= c[1]}
    OA = oracle.OMatrix.from_block_matrix(a)
    vals = U.values()
    rng = np.random.default_rng(8)
    picks = list(rng.choice(crow.shape[0], 12, replace=False)) + [0, crow.shape[0] - 1]
    for c in picks:
        ref, present = oracle.leaf_product(OA, OA, int(crow[c]), int(ccol[c]))
        assert present
        assert setref.rel_fro(vals[c].cpu().numpy(), ref) <= FP64_TOL

"""The sparse-product form of the boolean block product used by the
full-size tests equals the set definitions (every C leaf, its pair count)."""

from __future__ import annotations

import numpy as np
import pytest

from tests import setref


@pytest.mark.parametrize("grid,pa,pb,seed", [(7, 0.3, 0.4, 1), (33, 0.1, 0.2, 2),
                                             (64, 0.05, 0.05, 3), (5, 1.0, 1.0, 4),
                                             (9, 0.0, 0.5, 5)])
def test_product_pattern_counts_equal_the_set_definitions(grid, pa, pb, seed):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(seed)

    def pattern(p):
        m = rng.random((grid, grid)) < p
        r, c = np.nonzero(m)
        perm = rng.permutation(r.size)  # input order must not matter
        return r[perm], c[perm]

    ar, ac = pattern(pa)
    br, bc = pattern(pb)
    I, J, cnt = setref.product_pattern_counts(ar, ac, br, bc, grid)
    sa, sb = setref.pattern_set(ar, ac), setref.pattern_set(br, bc)
    per = setref.pairs_per_c_leaf(sa, sb)
    assert set(zip(I.tolist(), J.tolist())) == setref.boolean_product(sa, sb)
    assert {(i, j): n for i, j, n in zip(I.tolist(), J.tolist(), cnt.tolist())} == \
        {c: len(ks) for c, ks in per.items()}
    assert int(cnt.sum()) == setref.pair_count(sa, sb)
    key = I * grid + J
    assert np.all(np.diff(key) > 0)  # row-major, no repeats

"""Pins of the synthetic inputs against their stated recipes (no GPU): the
banded, 3D-locality, random and banded x 3D structures hold exactly the
leaves their definitions select (checked by brute force on the point
geometry), the generators are deterministic, and the workload sizes are the
documented ones (leaves, C leaves and leaf pairs by set logic)."""

from __future__ import annotations

import numpy as np
import pytest

import workloads as w
from tests import setref


def _sizes(a, b):
    pa, pb = setref.pattern_set(a.brow, a.bcol), setref.pattern_set(b.brow, b.bcol)
    return (len(pa), len(pb), len(setref.boolean_product(pa, pb)),
            setref.pair_count(pa, pb))


@pytest.mark.parametrize("n,sizes", [(8192, (5160, 5160, 12792, 226536)),
                                     (16384, (12056, 12056, 38392, 620344)),
                                     (32768, (28072, 28072, 111928, 1683176)),
                                     (65536, (60104, 60104, 259000, 3808840))])
def test_locality_sizes(n, sizes):
    a, b = w.config2(n)
    assert _sizes(a, b) == sizes
    assert a.b == 64 and a.n == n
    # A and B share the pattern and draw their values independently
    assert np.array_equal(a.brow, b.brow) and np.array_equal(a.bcol, b.bcol)
    assert not np.array_equal(a.vals[:4], b.vals[:4])


def test_banded_and_band_x_locality_sizes():
    assert _sizes(*w.config1()) == (1132, 1132, 2104, 10068)
    assert _sizes(*w.config5()) == (8632, 28072, 77210, 475064)


def test_banded_holds_exactly_the_band():
    a, _ = w.config1()
    g = a.n // a.b
    want = {(i, j) for i in range(g) for j in range(g) if abs(i - j) <= 4}
    assert setref.pattern_set(a.brow, a.bcol) == want
    assert np.all(np.abs(a.vals) <= 1.0) and a.vals.std() > 0.5


def test_locality_pattern_is_the_distance_rule():
    # brute force on sampled leaf pairs: stored iff the closest points of the
    # two 64-point groups are nearer than 6
    n, b, cutoff = 8192, 64, 6.0
    pts = w.lattice_points(n, w.structures.SEED_GEOM + 2)
    a, _ = w.config2(n)
    stored = setref.pattern_set(a.brow, a.bcol)
    g = n // b
    grp = pts.reshape(g, b, 3)
    rng = np.random.default_rng(17)
    cand = list(stored)
    picks = [cand[i] for i in rng.choice(len(cand), 150, replace=False)]
    picks += [tuple(int(v) for v in rng.integers(0, g, size=2)) for _ in range(150)]
    near = 0
    for i, j in picks:
        d = np.sqrt(((grp[i][:, None, :] - grp[j][None, :, :]) ** 2).sum(axis=2)).min()
        assert ((i, j) in stored) == (d < cutoff), (i, j, d)
        near += d < cutoff
    assert 150 <= near < len(picks)
    # the entries decay with the point distance: |a_pq| <= exp(-|x_p - x_q| / 2)
    k = 7
    i, j = int(a.brow[k]), int(a.bcol[k])
    dist = np.sqrt(((grp[i][:, None, :] - grp[j][None, :, :]) ** 2).sum(axis=2))
    assert np.all(np.abs(a.vals[k]) <= np.exp(-0.5 * dist) * (1 + 1e-12))


def test_lattice_is_a_jittered_morton_ordered_grid():
    pts = w.lattice_points(4096, 123)
    base = np.rint(pts)
    assert np.all(np.abs(pts - base) <= 0.25)
    # every lattice site of the first 16 x 16 x 16 Morton block appears once
    assert len({tuple(v) for v in base.astype(int)}) == 4096
    first = base[:64].astype(int)  # the first 4 x 4 x 4 sub-cube
    assert first.min() == 0 and first.max() == 3


def test_random_leaves_density_and_determinism():
    a, b = w.config3()
    g = a.n // a.b
    for m in (a, b):
        k = m.nblocks
        mean, sd = 0.01 * g * g, np.sqrt(0.01 * 0.99 * g * g)
        assert abs(k - mean) < 5 * sd
        assert abs(float(m.vals.mean())) < 0.01 and abs(float(m.vals.std()) - 1.0) < 0.01
    a2, _ = w.config3()
    assert np.array_equal(a.brow, a2.brow) and np.array_equal(a.vals, a2.vals)
    # A and B are independent draws
    assert setref.pattern_set(a.brow, a.bcol) != setref.pattern_set(b.brow, b.bcol)


def test_batched_products_follow_their_recipe():
    prods = w.batched_products(count=9, scale=0.125)
    kinds = [k for k, _, _ in prods]
    assert kinds == ["banded", "locality", "random"] * 3
    # the 64 sizes at 1/8 scale (the same draws): multiples of 64 in
    # [2048, 32768] / 8, log-uniform, so about half below the geometric mean
    full = w.batched_products(count=64, scale=0.125)
    sizes = [a.n for _, a, _ in full]
    assert all(s % 64 == 0 and 256 - 64 <= s <= 4096 for s in sizes)
    below = sum(s < 1024 for s in sizes)
    assert 16 <= below <= 48
    for kind, a, b in prods:
        assert a.b == 32 and b.b == 32 and a.n == b.n
        if kind == "banded":
            assert np.all(np.abs(a.brow.astype(int) - a.bcol.astype(int)) <= 4)
        elif kind == "locality":
            # 64-point groups split into 32-leaves: every 2 x 2 block of
            # 32-leaves of a stored 64-group pair is stored (zero quarters
            # would have been dropped only if all-zero)
            s = setref.pattern_set(a.brow, a.bcol)
            for i, j in list(s)[:50]:
                I, J = i // 2, j // 2
                assert {(2 * I + p, 2 * J + q) for p in (0, 1) for q in (0, 1)} <= s
            assert setref.pattern_set(b.brow, b.bcol) == s
        else:
            g = a.n // 32
            assert abs(a.nblocks - 0.02 * g * g) < 5 * np.sqrt(0.02 * g * g) + 1

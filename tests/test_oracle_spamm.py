"""Pins of the oracle's sparse approximate product (SpAMM): the recursion that
skips a quadrant product when the product of the quadrants' Frobenius norms
is below tau.  Checked against the exact product (tau = 0), the empty product
(tau above every norm product), the kept-pair set computed from leaf norms
with sets, a brute-force sum over the kept pairs, and the error bound given
by the dropped pairs."""

from __future__ import annotations

from collections import defaultdict

import numpy as np
import pytest

import oracle
import workloads as w
from tests import setref


def _leaf_norms(m):
    return {(int(r), int(c)): float(np.linalg.norm(v))
            for r, c, v in zip(m.brow, m.bcol, m.vals)}


def _pairs(na, nb):
    by_row = defaultdict(list)
    for (k, j), v in nb.items():
        by_row[k].append((j, v))
    out = []
    for (i, k), va in na.items():
        for j, vb in by_row.get(k, ()):
            out.append((i, k, j, va * vb))
    return out


def _matrices():
    pts = w.lattice_points(1024, 4011)
    pat = w.locality_pattern(pts, 8, 3.0)
    a = w.locality_matrix(pts, 8, 3.0, 11, pattern=pat)
    b = w.locality_matrix(pts, 8, 3.0, 12, pattern=pat)
    return a, b


def _safe_tau(prods, frac):
    """A threshold at the given quantile of the pair norm products, moved off
    any product by a relative margin so that rounding cannot flip a test."""
    vals = np.sort(np.array([p[3] for p in prods]))
    tau = float(np.quantile(vals, frac))
    while np.any(np.abs(vals - tau) <= 1e-9 * tau):
        tau *= 1.0 + 1e-6
    return tau


def test_tau_zero_is_the_exact_product():
    a, b = _matrices()
    A, B = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    C, n = A.multiply(B)
    S, ns = A.multiply_spamm(B, 0.0)
    assert n == ns
    assert np.array_equal(C.to_dense(), S.to_dense())
    assert C.pattern() == S.pattern()


def test_large_tau_is_nil():
    a, b = _matrices()
    A, B = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    S, ns = A.multiply_spamm(B, 1e30)
    assert ns == 0 and S.nleaves() == 0


@pytest.mark.parametrize("frac", [0.2, 0.5, 0.8])
def test_kept_pairs_sum_and_bound(frac):
    a, b = _matrices()
    A, B = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    prods = _pairs(_leaf_norms(a), _leaf_norms(b))
    tau = _safe_tau(prods, frac)
    S, ns = A.multiply_spamm(B, tau)
    kept = [p for p in prods if p[3] >= tau]
    dropped = [p for p in prods if p[3] < tau]
    assert ns == len(kept)
    assert S.pattern() == {(i, j) for i, _, j, _ in kept}
    # brute force: sum of the kept leaf products
    bs = a.b
    la = {(int(r), int(c)): v for r, c, v in zip(a.brow, a.bcol, a.vals)}
    lb = {(int(r), int(c)): v for r, c, v in zip(b.brow, b.bcol, b.vals)}
    ref = np.zeros((a.n, a.n))
    for i, k, j, _ in kept:
        ref[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] += la[(i, k)] @ lb[(k, j)]
    assert setref.rel_fro(S.to_dense(), ref) <= 1e-13
    # dropped pairs bound the error (triangle inequality, submultiplicativity)
    exact = a.to_dense() @ b.to_dense()
    err = float(np.linalg.norm(exact - S.to_dense()))
    assert err <= sum(p[3] for p in dropped) * (1 + 1e-12) + 1e-12


def test_monotone_in_tau():
    a, b = _matrices()
    A, B = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    counts = [A.multiply_spamm(B, t)[1] for t in (0.0, 0.1, 0.5, 1.0, 2.0, 5.0)]
    assert all(x >= y for x, y in zip(counts, counts[1:]))
    assert counts[0] > counts[-1]


def _spamm_pins_hold(mutant: int) -> bool:
    """The pins above, run on an oracle build with one planted mistake."""
    a, b = _matrices()
    A = oracle.OMatrix.from_block_matrix(a, mutant)
    B = oracle.OMatrix.from_block_matrix(b, mutant)
    prods = _pairs(_leaf_norms(a), _leaf_norms(b))
    for frac in (0.2, 0.5, 0.8):
        tau = _safe_tau(prods, frac)
        S, ns = A.multiply_spamm(B, tau)
        kept = [p for p in prods if p[3] >= tau]
        if ns != len(kept) or S.pattern() != {(i, j) for i, _, j, _ in kept}:
            return False
    return True


def test_spamm_pins_catch_a_planted_mistake():
    # mutant 8 compares the product of the squared norms with tau
    assert _spamm_pins_hold(0)
    assert not _spamm_pins_hold(8)

"""Pins of the oracle's upper-triangle product (the symmetric square C = A^2
of a symmetric A, paper Section 2.2): its leaves (I, J), I <= J, mirrored to
the full matrix, against numpy's dense product; its pattern and pair count
against the set definitions restricted to I <= J; and a planted mistake
(the quadrants above the diagonal also cut to their upper leaves) that these
pins catch."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import setref


def _mirror_dense(upper: np.ndarray, n: int, b: int) -> np.ndarray:
    """The symmetric matrix whose leaves on and above the diagonal are those
    of ``upper`` (which holds no leaf below it)."""
    g = n // b
    out = upper.copy()
    for i in range(g):
        for j in range(i):
            out[i * b:(i + 1) * b, j * b:(j + 1) * b] = upper[j * b:(j + 1) * b,
                                                              i * b:(i + 1) * b].T
    return out


def _cases():
    pts = w.lattice_points(512, 77)
    return [
        ("random", w.symmetrize(w.random_blocks(64, 4, 0.3, 5, dist="uniform"))),
        ("banded", w.symmetrize(w.banded(96, 8, 2, 6))),
        ("locality", w.symmetrize(w.locality_matrix(pts, 8, 3.0, 7))),
    ]


@pytest.mark.parametrize("name,a", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_upper_product_is_the_symmetric_square(name, a):
    dense = a.to_dense()
    assert np.array_equal(dense, dense.T)
    A = oracle.OMatrix.from_block_matrix(a)
    U, npairs = A.multiply_upper(A)
    pa = setref.pattern_set(a.brow, a.bcol)
    full = setref.boolean_product(pa, pa)
    assert U.pattern() == {(i, j) for i, j in full if i <= j}
    per = setref.pairs_per_c_leaf(pa, pa)
    assert npairs == sum(len(ks) for (i, j), ks in per.items() if i <= j)
    ref = dense @ dense
    assert setref.rel_fro(_mirror_dense(U.to_dense(), a.n, a.b), ref) <= 1e-13


def test_upper_pairs_about_half():
    a = w.symmetrize(w.banded(256, 8, 3, 9))
    A = oracle.OMatrix.from_block_matrix(a)
    _, nu = A.multiply_upper(A)
    _, nf = A.multiply(A)
    pa = setref.pattern_set(a.brow, a.bcol)
    per = setref.pairs_per_c_leaf(pa, pa)
    diag = sum(len(ks) for (i, j), ks in per.items() if i == j)
    # symmetric pattern: the pairs of (I, J) and (J, I) are equal in number
    assert 2 * nu - diag == nf


def test_nonsymmetric_upper_is_the_upper_part():
    x = w.random_blocks(64, 4, 0.3, 21, dist="uniform")
    y = w.random_blocks(64, 4, 0.3, 22, dist="uniform")
    X, Y = oracle.OMatrix.from_block_matrix(x), oracle.OMatrix.from_block_matrix(y)
    U, _ = X.multiply_upper(Y)
    ref = x.to_dense() @ y.to_dense()
    mask = np.kron(np.triu(np.ones((16, 16))), np.ones((4, 4)))
    got = U.to_dense()
    assert np.all(got[mask == 0] == 0)
    assert setref.rel_fro(got, ref * mask) <= 1e-13


def _pins_hold(mutant: int) -> bool:
    a = w.symmetrize(w.random_blocks(64, 4, 0.4, 31, dist="uniform"))
    A = oracle.OMatrix.from_block_matrix(a, mutant)
    U, _ = A.multiply_upper(A)
    d = a.to_dense()
    return setref.rel_fro(_mirror_dense(U.to_dense(), a.n, a.b), d @ d) <= 1e-13


def test_pins_catch_planted_mistake():
    assert _pins_hold(0)
    assert not _pins_hold(5)


def test_upper_pair_count_helper_by_brute_force():
    a = w.symmetrize(w.random_blocks(128, 4, 0.2, 41))
    pa = setref.pattern_set(a.brow, a.bcol)
    brute = sum(1 for (i, k) in pa for (k2, j) in pa if k == k2 and i <= j)
    assert setref.upper_pair_count(pa, pa) == brute

"""Pins of the oracle's matrix addition, addition of a scaled identity and
leaf truncation (paper, Section 2.2): against numpy's dense arithmetic (bit
for bit, since both form alpha*a + beta*b with separate roundings), the set
definitions of the patterns, the truncation's error bound and maximality
computed independently with numpy norms, and planted mistakes."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import setref


def _om(m, mutant=0):
    return oracle.OMatrix.from_block_matrix(m, mutant)


def _pair(seed, n=96, b=8, p=0.3):
    # n / b = 12: a grid that is not a power of two
    return (w.random_blocks(n, b, p, seed, dist="uniform"),
            w.random_blocks(n, b, p, seed + 1, dist="uniform"))


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (3.0, -2.0), (0.5, 0.0), (-1.25, 2.5)])
def test_add_is_the_dense_sum(alpha, beta):
    a, b = _pair(11)
    C = _om(a).add(alpha, _om(b), beta)
    assert np.array_equal(C.to_dense(), alpha * a.to_dense() + beta * b.to_dense())
    assert C.pattern() == setref.pattern_set(a.brow, a.bcol) | setref.pattern_set(b.brow, b.bcol)


def test_add_keeps_cancelled_leaves():
    a, _ = _pair(12)
    C = _om(a).add(1.0, _om(a), -1.0)
    assert C.pattern() == setref.pattern_set(a.brow, a.bcol)
    assert not np.any(C.to_dense())


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.5), (-2.0, 3.0)])
def test_add_identity(alpha, beta):
    a, _ = _pair(13)
    C = _om(a).add_identity(alpha, beta)
    ref = alpha * a.to_dense() + beta * np.eye(a.n)
    assert np.array_equal(C.to_dense(), ref)
    g = a.n // a.b
    assert C.pattern() == setref.pattern_set(a.brow, a.bcol) | {(i, i) for i in range(g)}


def _fro_truncation_reference(m, eps):
    """Leaves sorted by numpy's squared norms (ties by Morton position), the
    longest prefix whose summed squared norms stay <= eps^2."""
    r, c = m.brow, m.bcol
    order = np.argsort(oracle.morton_key(r, c), kind="stable")
    n2 = np.array([float(np.sum(m.vals[i] ** 2)) for i in order])
    rank = np.lexsort((np.arange(n2.size), n2))
    s = np.cumsum(n2[rank])
    m_rm = int(np.searchsorted(s, eps * eps, side="right"))
    removed = {(int(r[order[i]]), int(c[order[i]])) for i in rank[:m_rm]}
    return removed, s, m_rm


@pytest.mark.parametrize("frac", [0.0, 0.05, 0.3, 0.9])
def test_frobenius_truncation(frac):
    a, _ = _pair(14)
    d = a.to_dense()
    total = float(np.linalg.norm(d))
    removed_ref, s, _ = _fro_truncation_reference(a, frac * total)
    eps = frac * total
    # keep eps away from the prefix sums so rounding cannot move the cut
    while np.any(np.abs(s - eps * eps) <= 1e-9 * max(eps * eps, 1e-300)):
        eps *= 1.0 + 1e-6
    removed_ref, _, _ = _fro_truncation_reference(a, eps)
    T, rem = _om(a).truncate(eps, 0)
    assert T.pattern() == setref.pattern_set(a.brow, a.bcol) - removed_ref
    err = float(np.linalg.norm(d - T.to_dense()))
    assert err <= eps * (1 + 1e-12) + 1e-300
    assert abs(rem - err) <= 1e-12 * max(err, 1e-300)
    # kept leaves are copies
    kept = T.to_dense()
    mask = kept != 0
    assert np.array_equal(kept[mask], d[mask])


def test_frobenius_truncation_is_maximal():
    a, _ = _pair(15)
    total = float(np.linalg.norm(a.to_dense()))
    eps = 0.4 * total
    removed, s, m_rm = _fro_truncation_reference(a, eps)
    T, _ = _om(a).truncate(eps, 0)
    nrem = a.nblocks - T.nleaves()
    assert nrem == m_rm == len(removed)
    # removing one more leaf (the next smallest) would exceed eps
    assert s[m_rm] > eps * eps


@pytest.mark.parametrize("eps", [0.0, 0.5, 0.9, 1.0])
def test_max_norm_truncation(eps):
    a, _ = _pair(16)
    T, rem = _om(a).truncate(eps, 1)
    mx = {(int(r), int(c)): float(np.max(np.abs(v))) for r, c, v in zip(a.brow, a.bcol, a.vals)}
    assert T.pattern() == {k for k, v in mx.items() if v > eps}
    dropped = [v for v in mx.values() if v <= eps]
    assert rem == (max(dropped) if dropped else 0.0)
    assert float(np.max(np.abs(a.to_dense() - T.to_dense()))) <= eps


def test_truncation_removes_zero_leaves_at_eps_zero():
    a, _ = _pair(17)
    A = _om(a)
    Z = A.add(1.0, A, -1.0)  # every leaf cancelled, all kept by the addition
    assert Z.nleaves() == A.nleaves()
    T, rem = Z.truncate(0.0, 0)
    assert T.nleaves() == 0 and rem == 0.0
    T1, _ = A.truncate(0.0, 0)
    assert T1.pattern() == A.pattern()


def test_truncation_rejects_negative_eps():
    a, _ = _pair(18)
    with pytest.raises(oracle.OracleError):
        _om(a).truncate(-1.0, 0)


def _pins_hold(mutant):
    a, b = _pair(19)
    if not np.array_equal(_om(a, mutant).add(3.0, _om(b, mutant), -2.0).to_dense(),
                          3.0 * a.to_dense() - 2.0 * b.to_dense()):
        return False
    eps = 0.3 * float(np.linalg.norm(a.to_dense()))
    removed, _, _ = _fro_truncation_reference(a, eps)
    T, _ = _om(a, mutant).truncate(eps, 0)
    return T.pattern() == setref.pattern_set(a.brow, a.bcol) - removed


def test_pins_catch_planted_mistakes():
    # 6 copies a one-sided leaf of the first operand without its scale,
    # 7 removes the largest leaves first
    assert _pins_hold(0)
    assert not _pins_hold(6)
    assert not _pins_hold(7)

"""Pins of the oracle's McWeeny purification step (X <- 3X^2 - 2X^3 with
upper-triangle truncation) and of the oracle's mirror: against numpy's dense
polynomial, the eigen-decomposition limit (the projector onto the eigenvalues
above 1/2), and the truncation's error bound."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from oracle import purify
from tests import setref


def _start(n=128, b=8, seed=5, p=0.4):
    h = w.symmetrize(w.random_blocks(n, b, p, seed, dist="uniform"))
    lo, hi = w.gershgorin_bounds(h)
    H = oracle.OMatrix.from_block_matrix(h)
    # spectrum of H mapped into [0, 1], reversed: X0 = (hi I - H) / (hi - lo)
    X0 = H.add_identity(-1.0 / (hi - lo), hi / (hi - lo))
    return h, lo, hi, X0


def test_gershgorin_bounds_enclose_the_spectrum():
    h, lo, hi, _ = _start()
    ev = np.linalg.eigvalsh(h.to_dense())
    assert lo <= ev.min() and ev.max() <= hi


def _mirror_pin_holds(mutant: int = 0) -> bool:
    a = w.random_blocks(64, 4, 0.4, 3, dist="uniform")
    up = a.brow <= a.bcol
    u = w.BlockMatrix(a.n, a.b, a.brow[up], a.bcol[up], a.vals[up])
    d = u.to_dense()
    # element-level upper triangle, mirrored
    ref = np.triu(d) + np.triu(d, 1).T
    got = oracle.OMatrix.from_block_matrix(u, mutant).mirror_upper().to_dense()
    return bool(np.array_equal(got, ref))


def test_mirror_upper_of_the_oracle():
    assert _mirror_pin_holds()
    a = w.random_blocks(64, 4, 0.4, 3, dist="uniform")
    with pytest.raises(oracle.OracleError):
        oracle.OMatrix.from_block_matrix(a).mirror_upper()


def test_mirror_pin_catches_a_planted_mistake():
    # mutant 9 leaves the diagonal leaves unmirrored
    assert not _mirror_pin_holds(9)


def test_step_without_truncation_is_the_polynomial():
    _, _, _, X0 = _start()
    x = X0.to_dense()
    X1, removed, pairs = purify.mcweeny_step(X0, 0.0)
    assert removed == 0.0 and pairs > 0
    ref = 3.0 * x @ x - 2.0 * x @ x @ x
    assert setref.rel_fro(X1.to_dense(), ref) <= 1e-13


def test_iteration_converges_to_the_projector():
    h = w.symmetrize(w.random_blocks(64, 8, 1.0, 7, dist="uniform"))
    hv = np.linalg.eigvalsh(h.to_dense())
    lo, hi = float(hv[0]), float(hv[-1])
    X = oracle.OMatrix.from_block_matrix(h).add_identity(-1.0 / (hi - lo), hi / (hi - lo))
    x0 = X.to_dense()
    ev, vec = np.linalg.eigh(x0)
    assert np.all(np.abs(ev - 0.5) > 1e-3)
    proj = vec[:, ev > 0.5] @ vec[:, ev > 0.5].T
    for _ in range(80):
        X, _, _ = purify.mcweeny_step(X, 0.0)
    x = X.to_dense()
    assert float(np.linalg.norm(x @ x - x)) <= 1e-9
    assert abs(np.trace(x) - int(np.sum(ev > 0.5))) <= 1e-9
    assert float(np.linalg.norm(x - proj)) <= 1e-8


@pytest.mark.parametrize("eps", [1e-3, 1e-2, 1e-1])
def test_truncation_error_within_eps(eps):
    _, _, _, X0 = _start(n=256, b=8, seed=9, p=0.15)
    exact, _, _ = purify.mcweeny_step(X0, 0.0)
    trunc, removed, _ = purify.mcweeny_step(X0, eps)
    err = float(np.linalg.norm(exact.to_dense() - trunc.to_dense()))
    assert err <= eps * (1 + 1e-12)
    # the upper triangle lost `removed`; the full matrix loses between that
    # and sqrt(2) times that
    assert removed * (1 - 1e-12) <= err <= np.sqrt(2.0) * removed * (1 + 1e-12)
    d = trunc.to_dense()
    assert np.array_equal(d, d.T)


def test_step_is_the_composition_of_the_oracle_calls():
    _, _, _, X0 = _start(n=128, b=8, seed=11, p=0.3)
    eps = 0.05
    X1, removed, pairs = purify.mcweeny_step(X0, eps)
    x2u, p1 = X0.multiply_upper(X0)
    x3u, p2 = x2u.mirror_upper().multiply_upper(X0)
    tu, rem = x2u.add(3.0, x3u, -2.0).truncate(eps / np.sqrt(2.0), 0)
    assert pairs == p1 + p2 and removed == rem
    assert np.array_equal(X1.to_dense(), tu.mirror_upper().to_dense())


# ------------------------------------------------------- planted mistakes --
# Plausible mistakes in the step, planted in the oracle on the CPU; the pins
# against mathematics (the dense polynomial, the truncation bound) catch each.
# The composition test above is left out: it restates the step.

def _swapped_coefficients(X, eps):
    x2u, p1 = X.multiply_upper(X)
    x3u, p2 = x2u.mirror_upper().multiply_upper(X)
    tu, removed = x2u.add(2.0, x3u, -3.0).truncate(eps / np.sqrt(2.0), 0)
    return tu.mirror_upper(), removed, p1 + p2


def _full_eps_on_the_triangle(X, eps):
    x2u, p1 = X.multiply_upper(X)
    x3u, p2 = x2u.mirror_upper().multiply_upper(X)
    tu, removed = x2u.add(3.0, x3u, -2.0).truncate(eps, 0)
    return tu.mirror_upper(), removed, p1 + p2


def _unmirrored_square(X, eps):
    x2u, p1 = X.multiply_upper(X)
    x3u, p2 = x2u.multiply_upper(X)
    tu, removed = x2u.add(3.0, x3u, -2.0).truncate(eps / np.sqrt(2.0), 0)
    return tu.mirror_upper(), removed, p1 + p2


def _purify_pins_hold() -> bool:
    try:
        test_step_without_truncation_is_the_polynomial()
        for eps in (1e-3, 1e-2, 1e-1):
            test_truncation_error_within_eps(eps)
    except AssertionError:
        return False
    return True


def test_purify_pins_hold_unmutated():
    assert _purify_pins_hold()


@pytest.mark.parametrize("mutant", [_swapped_coefficients, _full_eps_on_the_triangle,
                                    _unmirrored_square])
def test_purify_pins_catch_planted_mistakes(monkeypatch, mutant):
    monkeypatch.setattr(purify, "mcweeny_step", mutant)
    assert not _purify_pins_hold()

"""GPU sparse approximate product: the SpAMM plan (pairs with leaf norm
product below tau dropped) against the oracle's SpAMM recursion; pattern and
pair counts bit-exact, values within the FP64 (and split) tolerance."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


def _safe_tau(a, b, frac):
    na = {(int(r), int(c)): float(np.linalg.norm(v)) for r, c, v in zip(a.brow, a.bcol, a.vals)}
    nb = {}
    for r, c, v in zip(b.brow, b.bcol, b.vals):
        nb.setdefault(int(r), []).append(float(np.linalg.norm(v)))
    prods = np.sort(np.array([va * vb for (i, k), va in na.items() for vb in nb.get(k, ())]))
    tau = float(np.quantile(prods, frac))
    while np.any(np.abs(prods - tau) <= 1e-9 * tau):
        tau *= 1.0 + 1e-6
    return tau


@pytest.mark.parametrize("name,frac", [("locality", 0.3), ("locality", 0.7),
                                       ("random", 0.5)])
def test_spamm_plan_matches_oracle(lib, name, frac):
    if name == "locality":
        a, b = w.config2(8192)
    else:
        a = w.random_blocks(2048, 32, 0.08, 51)
        b = w.random_blocks(2048, 32, 0.08, 52)
    tau = _safe_tau(a, b, frac)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply_spamm(A, B, tau)
    OA, OB = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    OS, npairs = OA.multiply_spamm(OB, tau)
    assert plan.npairs == npairs
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    gu.assert_same_pattern(C, OS)
    gu.assert_values_close(C, OS, 1e-13)
    Cs, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
    gu.assert_values_close(Cs, OS, 1e-11, leaf_tol=None)


def test_spamm_tau_zero_equals_exact_plan(lib):
    a, b = w.config1(2048, 32, 4)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    p0 = lib.cht_symbolic_multiply(A, B)
    ps = lib.cht_symbolic_multiply_spamm(A, B, 0.0)
    x, y = p0.arrays(), ps.arrays()
    for k in ("cseg", "pair_a", "pair_b", "crow", "ccol"):
        assert np.array_equal(x[k].numpy(), y[k].numpy()), k
    with pytest.raises(lib.ChtError):
        lib.cht_symbolic_multiply_spamm(A, B, -1.0)

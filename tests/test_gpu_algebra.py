"""GPU addition, addition of a scaled identity and truncation against the
oracle: patterns bit-exact, values bit-exact (both sides round alpha*a and
beta*b and their sum separately), truncation decisions identical for
thresholds kept away from the rounding-sensitive cut points; plus one and
two McWeeny purification steps (FP64 and split products) against the
oracle's step."""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


def _pair(name):
    if name == "locality":
        a, b = w.config2(8192)
        return a, b
    if name == "random":
        return w.random_blocks(2048, 32, 0.05, 81), w.random_blocks(2048, 32, 0.05, 82)
    # different patterns, grid not a power of two
    return w.banded(96 * 32, 32, 3, 83), w.random_blocks(96 * 32, 32, 0.02, 84)


def _assert_bitwise(M, omat):
    gu.assert_same_pattern(M, omat)
    _, _, gv = gu.host_leaves(M)
    _, _, ov = omat.leaves()
    assert np.array_equal(gv, ov)


@pytest.mark.parametrize("name", ["locality", "random", "mixed"])
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (3.0, -2.0), (-0.3, 0.7)])
def test_add_bit_exact(lib, name, alpha, beta):
    a, b = _pair(name)
    C = lib.cht_add(alpha, gu.upload(lib, a), beta, gu.upload(lib, b))
    OA, OB = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    _assert_bitwise(C, OA.add(alpha, OB, beta))


@pytest.mark.parametrize("name", ["locality", "mixed"])
def test_add_identity_bit_exact(lib, name):
    a, _ = _pair(name)
    for alpha, beta in ((1.0, 1.0), (-0.25, 0.75)):
        C = lib.cht_add_identity(alpha, gu.upload(lib, a), beta)
        _assert_bitwise(C, oracle.OMatrix.from_block_matrix(a).add_identity(alpha, beta))


def test_add_edge_cases(lib):
    a, _ = _pair("random")
    A = gu.upload(lib, a)
    Z = lib.cht_add(1.0, A, -1.0, A)  # cancelled leaves stay stored
    assert Z.nblocks == A.nblocks and not bool(Z.values().any())
    e = w.BlockMatrix(a.n, a.b, np.zeros(0, np.int32), np.zeros(0, np.int32),
                      np.zeros((0, a.b, a.b)))
    E = gu.upload(lib, e)
    assert lib.cht_add(1.0, E, 1.0, E).nblocks == 0
    _assert_bitwise(lib.cht_add(2.0, E, 1.0, A),
                    oracle.OMatrix.from_block_matrix(e).add(2.0, oracle.OMatrix.from_block_matrix(a), 1.0))
    eye = lib.cht_add_identity(1.0, E, 1.0)
    assert eye.nblocks == a.grid
    assert np.array_equal(eye.to_dense().cpu().numpy(), np.eye(a.n))
    other = gu.upload(lib, w.random_blocks(1024, 32, 0.1, 85))
    with pytest.raises(lib.ChtError):
        lib.cht_add(1.0, A, 1.0, other)


def _safe_fro_eps(m, frac):
    """eps at frac of the total norm, moved off every prefix sum of the
    sorted squared leaf norms by a relative margin."""
    n2 = np.sort(np.array([float(np.sum(v * v)) for v in m.vals]))
    s = np.cumsum(n2)
    eps = frac * math.sqrt(float(s[-1]))
    while np.any(np.abs(s - eps * eps) <= 1e-9 * eps * eps):
        eps *= 1.0 + 1e-6
    return eps


@pytest.mark.parametrize("name", ["locality", "random"])
@pytest.mark.parametrize("frac", [0.01, 0.1, 0.5])
def test_truncate_frobenius_matches_oracle(lib, name, frac):
    a, _ = _pair(name)
    eps = _safe_fro_eps(a, frac)
    T, removed = lib.cht_truncate(gu.upload(lib, a), eps, lib.CHT_TRUNC_FRO)
    OT, orem = oracle.OMatrix.from_block_matrix(a).truncate(eps, 0)
    _assert_bitwise(T, OT)
    assert removed <= eps
    assert abs(removed - orem) <= 1e-12 * max(orem, 1e-300)


@pytest.mark.parametrize("rel", [0.0, 1e-3, 0.05, 0.5])
def test_truncate_max_matches_oracle(lib, rel):
    a, _ = _pair("locality")
    eps = rel * float(np.max(np.abs(a.vals)))
    T, removed = lib.cht_truncate(gu.upload(lib, a), eps, lib.CHT_TRUNC_MAX)
    OT, orem = oracle.OMatrix.from_block_matrix(a).truncate(eps, 1)
    _assert_bitwise(T, OT)
    assert removed == orem


def test_truncate_edge_cases(lib):
    a, _ = _pair("random")
    A = gu.upload(lib, a)
    Z = lib.cht_add(1.0, A, -1.0, A)
    T0, r0 = lib.cht_truncate(Z, 0.0)
    assert T0.nblocks == 0 and r0 == 0.0
    T1, r1 = lib.cht_truncate(A, 0.0)
    assert T1.nblocks == A.nblocks and r1 == 0.0
    Tall, rall = lib.cht_truncate(A, 1e300)
    assert Tall.nblocks == 0
    assert abs(rall - float(np.linalg.norm(a.vals))) <= 1e-12 * rall
    with pytest.raises(lib.ChtError):
        lib.cht_truncate(A, -1.0)
    with pytest.raises(lib.ChtError):
        lib.cht_truncate(A, float("nan"))
    with pytest.raises(lib.ChtError):
        lib.cht_truncate(A, 1.0, 7)


def _purification_start(n, b):
    h = w.config2_symmetric(n, b)
    lo, hi = w.gershgorin_bounds(h)
    return h, -1.0 / (hi - lo), hi / (hi - lo)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_mcweeny_steps_match_oracle(lib, mode):
    from paper_2011_11762_gb300 import purify
    h, alpha, beta = _purification_start(4096, 32)
    X = lib.cht_add_identity(alpha, gu.upload(lib, h), beta)
    OX = oracle.OMatrix.from_block_matrix(h).add_identity(alpha, beta)
    gmode = lib.CHT_FP64 if mode == "fp64" else lib.CHT_SPLIT_BF16
    tol = 1e-13 if mode == "fp64" else 1e-11
    for _ in range(2):
        # the oracle's step (the composition in oracle.purify), with the
        # threshold moved off the cut points of its truncation
        x2u, p1 = OX.multiply_upper(OX)
        x3u, p2 = x2u.mirror_upper().multiply_upper(OX)
        yu = x2u.add(3.0, x3u, -2.0)
        _, _, yv = yu.leaves()
        s = np.cumsum(np.sort(np.array([float(np.sum(v * v)) for v in yv])))
        eps = 1e-3 * math.sqrt(float(s[-1]))
        while np.any(np.abs(s - eps * eps / 2.0) <= 1e-7 * eps * eps):
            eps *= 1.0 + 1e-5
        tu, orem = yu.truncate(eps / math.sqrt(2.0), 0)
        OX = tu.mirror_upper()
        X, info = purify.mcweeny_step(X, eps, mode=gmode)
        assert info["pairs"] == p1 + p2
        gu.assert_same_pattern(X, OX)
        gu.assert_values_close(X, OX, tol, leaf_tol=None)
        assert abs(info["removed"] - orem) <= 1e-6 * max(orem, 1e-300)
        d = X.to_dense().cpu().numpy()
        assert np.array_equal(d, d.T)

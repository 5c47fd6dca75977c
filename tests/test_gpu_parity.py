"""GPU parity: symbolic phase bit-exact and FP64 numeric phase within 1e-13
relative Frobenius error of the CPU oracle, through the C ABI."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13


def _cases():
    return {
        # config 1 at full size: banded +-4, N = 4096, 32x32 leaves
        "banded_4096_b32": lambda: w.config1(),
        # non-power-of-two leaf grid with a ragged band
        "banded_1440_b32": lambda: w.config1(1440, 32, 3),
        # 3D locality, smallest member of the scaling sequence (b = 64)
        "locality_8192_b64": lambda: w.config2(8192),
        # random leaves (config 3 structure at reduced size)
        "random_4096_b32": lambda: (w.random_blocks(4096, 32, 0.03, 1003),
                                    w.random_blocks(4096, 32, 0.03, 2003)),
        # banded x 3D (config 5 structure at reduced size)
        "band_x_locality_8192_b64": lambda: (w.banded(8192, 64, 8, 1005),
                                             w.locality_matrix(w.lattice_points(8192, 4005),
                                                               64, 6.0, 2005)),
    }


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("engine", [0, 1, 2])
def test_multiply_matches_oracle(lib, name, engine):
    a, b = _cases()[name]()
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    Co, npairs = gu.oracle_product(a, b)
    assert plan.npairs == npairs
    assert plan.nnzb_C == Co.nleaves()
    lib.set_option(lib.OPT_FP64_ENGINE, engine)
    try:
        C, bound = lib.cht_multiply(plan, A, B, sync=True)
    finally:
        lib.set_option(lib.OPT_FP64_ENGINE, 1)
    gu.assert_same_pattern(C, Co)
    gu.assert_values_close(C, Co, FP64_TOL)
    assert 0 < bound < 1e-10


@pytest.mark.parametrize("name", ["banded_1440_b32", "random_4096_b32",
                                  "band_x_locality_8192_b64"])
def test_symbolic_pairs_bit_exact(lib, name):
    a, b = _cases()[name]()
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    arr = gu.check_plan_pairs(plan, a, b)
    pa = setref.pattern_set(a.brow, a.bcol)
    pb = setref.pattern_set(b.brow, b.bcol)
    assert plan.npairs == setref.pair_count(pa, pb)
    got = set(zip(arr["crow"].tolist(), arr["ccol"].tolist()))
    assert got == setref.boolean_product(pa, pb)
    keys = oracle.morton_key(arr["crow"].numpy(), arr["ccol"].numpy())
    assert np.all(np.diff(keys) > 0)  # C leaves in Morton order
    seglen = np.diff(arr["cseg"].numpy())
    assert np.all(np.diff(seglen[arr["order"].numpy()]) <= 0)  # longest first


def test_morton_schedule_option(lib):
    a, b = w.config1(2048, 32, 4)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    lib.set_option(lib.OPT_SCHEDULE, 1)
    try:
        plan = lib.cht_symbolic_multiply(A, B)
        C, _ = lib.cht_multiply(plan, A, B, sync=True)
    finally:
        lib.set_option(lib.OPT_SCHEDULE, 0)
    assert np.array_equal(plan.arrays()["order"].numpy(), np.arange(plan.nnzb_C))
    Co, _ = gu.oracle_product(a, b)
    gu.assert_values_close(C, Co, FP64_TOL)


def test_identity_products_bit_exact(lib):
    for bs in (32, 64):
        n = bs * 12
        a = w.random_blocks(n, bs, 0.3, 7 + bs, dist="uniform")
        g = n // bs
        eye = w.BlockMatrix(n, bs, np.arange(g, dtype=np.int32), np.arange(g, dtype=np.int32),
                            np.broadcast_to(np.eye(bs), (g, bs, bs)).copy())
        A, E = gu.upload(lib, a), gu.upload(lib, eye)
        for X, Y in ((A, E), (E, A)):
            plan = lib.cht_symbolic_multiply(X, Y)
            C, _ = lib.cht_multiply(plan, X, Y, sync=True)
            assert np.array_equal(C.to_dense().cpu().numpy(), a.to_dense())


def test_results_bitwise_reproducible(lib):
    a, b = w.config2(8192)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C1, _ = lib.cht_multiply(plan, A, B, sync=True)
    v1 = C1.values().clone()
    C2, _ = lib.cht_multiply(plan, A, B, out=C1, sync=True)
    assert C2 is C1
    assert bool((C1.values() == v1).all())


def test_empty_and_zero_operands(lib):
    a = w.banded(1024, 32, 2, 21)
    empty = w.BlockMatrix(1024, 32, np.zeros(0, np.int32), np.zeros(0, np.int32),
                          np.zeros((0, 32, 32)))
    zeros = w.BlockMatrix(1024, 32, a.brow.copy(), a.bcol.copy(), np.zeros_like(a.vals))
    A = gu.upload(lib, a)
    for z in (empty, zeros):
        Z = gu.upload(lib, z)
        assert Z.nblocks == 0
        for X, Y in ((A, Z), (Z, A), (Z, Z)):
            plan = lib.cht_symbolic_multiply(X, Y)
            assert plan.npairs == 0 and plan.nnzb_C == 0
            C, _ = lib.cht_multiply(plan, X, Y, sync=True)
            assert C.nblocks == 0
            assert float(C.to_dense().abs().max()) == 0.0


def test_single_leaf_and_tiny_grid(lib):
    for n, bs in ((32, 32), (64, 64), (96, 32)):
        a = w.random_blocks(n, bs, 1.0, 31, dist="uniform")
        b = w.random_blocks(n, bs, 1.0, 32, dist="uniform")
        A, B = gu.upload(lib, a), gu.upload(lib, b)
        plan = lib.cht_symbolic_multiply(A, B)
        C, _ = lib.cht_multiply(plan, A, B, sync=True)
        ref = a.to_dense() @ b.to_dense()
        assert setref.rel_fro(C.to_dense().cpu().numpy(), ref) <= FP64_TOL


def test_zero_leaves_are_dropped(lib):
    a = w.banded(2048, 32, 3, 41)
    a.vals[5] = 0.0
    a.vals[17] = 0.0
    A = gu.upload(lib, a)
    assert A.nblocks == a.nblocks - 2
    br, bc, vals = gu.host_leaves(A)
    O = oracle.OMatrix.from_block_matrix(a)
    orow, ocol, ov = O.leaves()
    assert np.array_equal(br, orow) and np.array_equal(bc, ocol)
    assert np.array_equal(vals, ov)


def test_to_dense_round_trip(lib):
    a = w.random_blocks(2048, 64, 0.1, 51)
    A = gu.upload(lib, a)
    assert np.array_equal(A.to_dense().cpu().numpy(), a.to_dense())


def test_associativity(lib):
    a = w.banded(2048, 32, 3, 61)
    b = w.random_blocks(2048, 32, 0.05, 62, dist="uniform")
    c = w.banded(2048, 32, 2, 63)
    A, B, C = (gu.upload(lib, m) for m in (a, b, c))
    AB, _ = lib.cht_multiply(lib.cht_symbolic_multiply(A, B), A, B)
    BC, _ = lib.cht_multiply(lib.cht_symbolic_multiply(B, C), B, C)
    L, _ = lib.cht_multiply(lib.cht_symbolic_multiply(AB, C), AB, C, sync=True)
    R, _ = lib.cht_multiply(lib.cht_symbolic_multiply(A, BC), A, BC, sync=True)
    lr, lc, lv = gu.host_leaves(L)
    rr, rc, rv = gu.host_leaves(R)
    assert np.array_equal(lr, rr) and np.array_equal(lc, rc)
    assert setref.rel_fro(lv, rv) <= 1e-12


def test_invalid_inputs_are_rejected(lib):
    import torch
    a = w.banded(1024, 32, 1, 71)
    br = torch.from_numpy(np.r_[a.brow, a.brow[:1]])
    bc = torch.from_numpy(np.r_[a.bcol, a.bcol[:1]])
    vals = torch.from_numpy(np.concatenate([a.vals, a.vals[:1]]))
    with pytest.raises(lib.ChtError) as e:
        lib.cht_mat_from_blocks(1024, 32, br, bc, vals)
    assert e.value.code == lib.CHT_ERR_DUPLICATE
    with pytest.raises(lib.ChtError) as e:
        lib.cht_mat_from_blocks(1024, 32, torch.tensor([32], dtype=torch.int32),
                                torch.tensor([0], dtype=torch.int32),
                                torch.ones(1, 32, 32, dtype=torch.float64))
    assert e.value.code == lib.CHT_ERR_INVALID
    with pytest.raises(lib.ChtError) as e:
        lib.cht_mat_from_blocks(1000, 32, torch.from_numpy(a.brow), torch.from_numpy(a.bcol),
                                torch.from_numpy(a.vals))
    assert e.value.code == lib.CHT_ERR_INVALID
    A = gu.upload(lib, a)
    B64 = gu.upload(lib, w.banded(1024, 64, 1, 72))
    with pytest.raises(lib.ChtError) as e:
        lib.cht_symbolic_multiply(A, B64)
    assert e.value.code == lib.CHT_ERR_SHAPE


def test_bounded_wait_reports_timeout(lib):
    # A zero wait budget makes every bounded device-side wait give up at once:
    # the kernel records the timeout, drains its copies and returns; the
    # context stays usable.
    a, b = w.config1(1024, 32, 2)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    old = lib.get_option(lib.OPT_WAIT_BUDGET_NS)
    lib.set_option(lib.OPT_WAIT_BUDGET_NS, 0)
    try:
        with pytest.raises(lib.ChtError) as e:
            lib.cht_multiply(plan, A, B, sync=True)
        assert e.value.code == lib.CHT_ERR_TIMEOUT
    finally:
        lib.set_option(lib.OPT_WAIT_BUDGET_NS, old)
    lib.sync_status()
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    Co, _ = gu.oracle_product(a, b)
    gu.assert_values_close(C, Co, FP64_TOL)


@pytest.fixture(scope="module")
def full3d(lib):
    """The benchmark workload: 3D locality, N = 65536, 64x64 leaves."""
    a, b = w.config2(65536)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    return a, b, A, B, lib.cht_symbolic_multiply(A, B)


def _shift_rows(m):
    """The same leaves with their leaf rows moved down by one (cyclically):
    as many leaves as m, on another pattern."""
    return w.BlockMatrix(m.n, m.b, ((m.brow + 1) % m.grid).astype(np.int32), m.bcol.copy(),
                         m.vals.copy())


def test_operands_checked_against_plan(lib):
    # The plan's pair lists index the leaves of its operands, so operands on
    # another pattern with the same leaf count are refused before any work;
    # a matrix rebuilt from the same blocks (another pattern object, the same
    # leaves) is accepted and gives the same product bit for bit.
    torch = pytest.importorskip("torch")
    a, b = w.config1(2048, 32, 4)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    As = gu.upload(lib, _shift_rows(a))
    Bs = gu.upload(lib, _shift_rows(b))
    assert As.nblocks == A.nblocks and Bs.nblocks == B.nblocks
    for x, y in ((As, B), (A, Bs), (As, Bs)):
        for mode in (lib.CHT_FP64, lib.CHT_SPLIT_BF16):
            with pytest.raises(lib.ChtError) as e:
                lib.cht_multiply(plan, x, y, mode=mode)
            assert e.value.code == lib.CHT_ERR_SHAPE
        with pytest.raises(lib.ChtError) as e:
            lib.cht_multiply(plan, x, y, out=C)  # an existing output is not touched either
        assert e.value.code == lib.CHT_ERR_SHAPE
        out = torch.empty((plan.nnzb_C, a.b, a.b), dtype=torch.float64, pin_memory=True)
        with pytest.raises(lib.ChtError) as e:
            lib.cht_multiply_to_host(plan, x, y, out)
        assert e.value.code == lib.CHT_ERR_SHAPE
        with pytest.raises(lib.ChtError) as e:
            lib.Batch([plan], [x], [y])
        assert e.value.code == lib.CHT_ERR_SHAPE
    ref = C.values().clone()
    A2, B2 = gu.upload(lib, a), gu.upload(lib, b)  # rebuilt: equal patterns
    for x, y in ((A2, B), (A, B2), (A2, B2)):
        C2, _ = lib.cht_multiply(plan, x, y, sync=True)
        assert torch.equal(C2.values(), ref)
    lib.sync_status()


def test_full_size_operands_checked_against_plan(lib, full3d):
    # On the benchmark workload A and B share one pattern (same lattice and
    # cutoff; only their values differ), so plan(A, B) applied to (B, A)
    # indexes stored leaves and is the product B*A: accepted, and equal bit
    # for bit to the product on plan(B, A).  A with its leaf rows shifted
    # has as many leaves (60104) on another pattern: refused.
    torch = pytest.importorskip("torch")
    a, b, A, B, plan = full3d
    assert A.nblocks == B.nblocks
    BA, _ = lib.cht_multiply(plan, B, A, sync=True)
    ref, _ = lib.cht_multiply(lib.cht_symbolic_multiply(B, A), B, A, sync=True)
    assert torch.equal(BA.values(), ref.values())
    del BA, ref
    As = gu.upload(lib, _shift_rows(a))
    assert As.nblocks == A.nblocks
    for x, y in ((As, B), (B, As)):
        with pytest.raises(lib.ChtError) as e:
            lib.cht_multiply(plan, x, y)
        assert e.value.code == lib.CHT_ERR_SHAPE


def test_full_size_3d_locality_sampled(lib, full3d):
    # N = 65536, 64x64 leaves (the benchmark workload): pattern counts exact,
    # sampled C leaves against the oracle's single-leaf product.
    a, b, A, B, plan = full3d
    pa = setref.pattern_set(a.brow, a.bcol)
    pb = setref.pattern_set(b.brow, b.bcol)
    assert plan.npairs == setref.pair_count(pa, pb)
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    arr = plan.arrays()
    crow, ccol = arr["crow"].numpy(), arr["ccol"].numpy()
    assert set(zip(crow.tolist(), ccol.tolist())) == setref.boolean_product(pa, pb)
    OA = oracle.OMatrix.from_block_matrix(a)
    OB = oracle.OMatrix.from_block_matrix(b)
    vals = C.values()
    seglen = np.diff(arr["cseg"].numpy())
    rng = np.random.default_rng(7)
    picks = list(rng.choice(crow.shape[0], 12, replace=False)) + [int(np.argmax(seglen)), 0,
                                                                 crow.shape[0] - 1]
    for c in picks:
        ref, present = oracle.leaf_product(OA, OB, int(crow[c]), int(ccol[c]))
        assert present
        got = vals[c].cpu().numpy()
        assert setref.rel_fro(got, ref) <= FP64_TOL


def test_dense_torch_cross_check(lib):
    # the whole product against a dense FP64 matmul (cuBLAS) of the densified
    # operands: N = 8192, 3D locality
    torch = pytest.importorskip("torch")
    a, b = w.config2(8192)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    ref = torch.matmul(A.to_dense(), B.to_dense())
    got = C.to_dense()
    rel = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
    assert rel <= FP64_TOL, rel
    # outside C's pattern the dense product is exactly zero
    crow, ccol = (t.long() for t in C.coords())
    mask = torch.zeros((a.grid, a.grid), dtype=torch.bool, device="cuda")
    mask[crow, ccol] = True
    full = torch.kron(mask.to(torch.float64), torch.ones((a.b, a.b), dtype=torch.float64,
                                                         device="cuda")) != 0
    assert not bool(ref[~full].any())


@pytest.mark.parametrize("nchunks", [1, 3, 8])
def test_multiply_to_host_equals_device_product(lib, nchunks):
    # the chunked product streamed to pinned host memory equals the device
    # product bit for bit (same kernel, same per-leaf summation order)
    torch = pytest.importorskip("torch")
    a, b = w.config2(8192)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    out = torch.empty((plan.nnzb_C, a.b, a.b), dtype=torch.float64, pin_memory=True)
    out.fill_(float("nan"))
    lib.cht_multiply_to_host(plan, A, B, out, nchunks=nchunks)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(out, C.values().cpu())
    with pytest.raises(lib.ChtError):
        lib.cht_multiply_to_host(plan, A, B, out, nchunks=0)

"""Batched products in one persistent launch (FP64 and split forms), CUDA
graph capture of a batch run, and the leaf-size / schedule autotuner."""

from __future__ import annotations

import numpy as np
import pytest

import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


def _products(count=9, scale=0.12):
    return w.batched_products(count=count, scale=scale)


def _build(lib, prods, sizes):
    mats, plans = [], []
    for (kind, a, b), bs in zip(prods, sizes):
        if bs != a.b:
            a, b = w.reblock(a, bs), w.reblock(b, bs)
        A, B = gu.upload(lib, a), gu.upload(lib, b)
        mats.append((A, B, a, b))
        plans.append(lib.cht_symbolic_multiply(A, B))
    return mats, plans


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_batch_matches_single_products(lib, mode):
    prods = _products()
    sizes = [32 if i % 2 else 64 for i in range(len(prods))]
    mats, plans = _build(lib, prods, sizes)
    m = lib.CHT_FP64 if mode == "fp64" else lib.CHT_SPLIT_BF16
    bt = lib.Batch(plans, [x[0] for x in mats], [x[1] for x in mats], mode=m)
    bt.run()
    lib.sync_status()
    for i, ((A, B, a, b), plan) in enumerate(zip(mats, plans)):
        single, _ = lib.cht_multiply(plan, A, B, mode=m, sync=True)
        out = bt.output(i)
        assert out.nblocks == plan.nnzb_C
        got, ref = out.values(), single.values()
        if mode == "fp64":
            assert bool((got == ref).all()), i  # same kernel arithmetic, same order
        else:
            assert setref.rel_fro(got.cpu().numpy(), ref.cpu().numpy()) == 0.0, i
        Co, _ = gu.oracle_product(a, b)
        gu.assert_same_pattern(out, Co)
        gu.assert_values_close(out, Co, 1e-13 if mode == "fp64" else 1e-12,
                                 leaf_tol=1e-13 if mode == "fp64" else None)


def test_batch_in_cuda_graph(lib):
    import torch
    prods = _products(count=6)
    mats, plans = _build(lib, prods, [64, 32, 64, 32, 32, 64])
    for m in (lib.CHT_FP64, lib.CHT_SPLIT_BF16):
        bt = lib.Batch(plans, [x[0] for x in mats], [x[1] for x in mats], mode=m)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            bt.run(stream=s)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        ref = [bt.output(i).values().clone() for i in range(len(plans))]
        for i in range(len(plans)):
            bt.output(i).values().fill_(float("nan"))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bt.run()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        lib.sync_status()
        for i in range(len(plans)):
            assert bool((bt.output(i).values() == ref[i]).all())


def test_autotuner_picks_valid_blockings(lib, tmp_path):
    import torch

    from paper_2011_11762_gb300 import autotune
    prods = _products(count=6)
    spec = [(a.n, (torch.from_numpy(a.brow), torch.from_numpy(a.bcol), torch.from_numpy(a.vals)),
             (torch.from_numpy(b.brow), torch.from_numpy(b.bcol), torch.from_numpy(b.vals)))
            for _, a, b in prods]
    cache = str(tmp_path / "tune.json")
    tuned = autotune.tune(spec, mode=lib.CHT_FP64, cache_path=cache)
    assert len(tuned.leaf_sizes) == len(prods)
    assert set(tuned.leaf_sizes) <= {32, 64}
    assert tuned.schedule in ("longest-first", "morton")
    tuned.batch.run()
    lib.sync_status()
    for i, (_, a, b) in enumerate(prods):
        out = tuned.batch.output(i)
        ref = a.to_dense() @ b.to_dense()
        assert setref.rel_fro(out.to_dense().cpu().numpy(), ref) <= 1e-13
    # second run reads the cache: same choices, no re-timing
    again = autotune.tune(spec, mode=lib.CHT_FP64, cache_path=cache)
    assert again.leaf_sizes == tuned.leaf_sizes
    assert all(len(t) == 1 for t in again.timings["per_product_ms"])


def test_reblock_preserves_the_matrix(lib):
    import torch

    from paper_2011_11762_gb300 import autotune
    a = w.random_blocks(512, 32, 0.1, 77)
    r, c, v = autotune.reblock(512, 32, torch.from_numpy(a.brow), torch.from_numpy(a.bcol),
                               torch.from_numpy(a.vals), 64)
    M = lib.cht_mat_from_blocks(512, 64, r, c, v)
    assert np.array_equal(M.to_dense().cpu().numpy(), a.to_dense())
    ref = w.reblock(a, 64)
    assert M.nblocks == ref.nblocks


def test_split_batch_with_long_segments(lib):
    # a product whose leaf (0, 0) sums more pairs than one unit may, batched
    # with ordinary ones: it is computed in pieces inside the batch, and the
    # batch (also in a graph replay) equals the single products
    import torch
    a1, b1 = w.dense_line_pair(1100 * 64, 64, 1, 93)
    a2, b2 = w.dense_line_pair(4100 * 32, 32, 1, 95)
    mats = [(gu.upload(lib, a), gu.upload(lib, b), a, b)
            for a, b in ((a1, b1), (a2, b2), *[(x[1], x[2]) for x in _products(3)])]
    plans = [lib.cht_symbolic_multiply(A, B) for A, B, _, _ in mats]
    bt = lib.Batch(plans, [x[0] for x in mats], [x[1] for x in mats], mode=lib.CHT_SPLIT_BF16)
    bt.run()
    lib.sync_status()
    for i, ((A, B, a, b), plan) in enumerate(zip(mats, plans)):
        single, _ = lib.cht_multiply(plan, A, B, mode=lib.CHT_SPLIT_BF16, sync=True)
        assert bool((bt.output(i).values() == single.values()).all()), i
        if i < 2:
            Co, _ = gu.oracle_product(a, b)
            gu.assert_values_close(bt.output(i), Co, 1e-11, leaf_tol=None)
    ref = [bt.output(i).values().clone() for i in range(len(plans))]
    for i in range(len(plans)):
        bt.output(i).values().fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bt.run()
    g.replay()
    torch.cuda.synchronize()
    lib.sync_status()
    for i in range(len(plans)):
        assert bool((bt.output(i).values() == ref[i]).all()), i

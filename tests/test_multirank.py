"""The multi-rank path on CPU with gloo (world size 2): the C-leaf partition
covers every leaf exactly once and balances pairs, ranks computing their
ranges (here with the CPU oracle's single-leaf product) reassemble the whole
product, and the timing / total helpers reduce across ranks."""

from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_2011_11762_gb300 import shard


def test_partition_covers_and_balances():
    rng = np.random.default_rng(3)
    lens = rng.integers(1, 40, size=1000)
    for nr in (1, 2, 3, 8):
        parts = shard.partition_units(lens, nr)
        assert parts[0][0] == 0 and parts[-1][1] == lens.shape[0]
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        loads = [int(lens[lo:hi].sum()) for lo, hi in parts]
        assert max(loads) - min(loads) <= 2 * int(lens.max())
    assert shard.partition_units([], 2) == [(0, 0), (0, 0)]
    assert sum(hi - lo for lo, hi in shard.partition_units([5], 3)) == 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_q):
    import torch.distributed as dist

    import oracle
    import workloads as w
    from paper_2011_11762_gb300 import shard as sh
    from tests import setref

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = w.config1(1024, 32, 3)
        A = oracle.OMatrix.from_block_matrix(a)
        B = oracle.OMatrix.from_block_matrix(b)
        pa, pb = setref.pattern_set(a.brow, a.bcol), setref.pattern_set(b.brow, b.bcol)
        segs = setref.pairs_per_c_leaf(pa, pb)
        keys = sorted(segs, key=lambda ij: int(oracle.morton_key([ij[0]], [ij[1]])[0]))
        lens = [len(segs[k]) for k in keys]
        lo, hi = sh.partition_units(lens, world)[rank]
        mine = {}
        for I, J in keys[lo:hi]:
            v, present = oracle.leaf_product(A, B, I, J)
            assert present
            mine[(I, J)] = v
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        slowest = sh.max_over_ranks(float(rank + 1))
        total = sh.sum_over_ranks(float(sum(lens[lo:hi])))
        if rank == 0:
            full = {}
            for part in gathered:
                assert not (set(part) & set(full))  # every leaf owned once
                full.update(part)
            C = A @ B
            cr, cc, cv = C.leaves()
            assert set(full) == set(zip(cr.tolist(), cc.tolist()))
            err = max(setref.rel_fro(full[(int(r), int(c))], cv[i])
                      for i, (r, c) in enumerate(zip(cr, cc)))
            out_q.put(("ok", err, slowest, total, sum(lens)))
    except Exception as e:  # report to the parent
        out_q.put(("error", repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_product():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = q.get(timeout=10)
    assert res[0] == "ok", res
    _, err, slowest, total, want = res
    assert err <= 1e-13
    assert slowest == 2.0
    assert total == want
    _ = torch

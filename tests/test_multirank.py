"""The multi-rank path on CPU with gloo: the C-leaf partition covers every
leaf exactly once and balances pairs, ranks computing their ranges (here
with the CPU oracle's single-leaf product) reassemble the whole product, and
the timing / total helpers reduce across ranks.  With distributed operands
(each rank starting with one Morton range of A's and of B's leaves), the
ranks exchange exactly the leaves their pairs use, point to point, and still
reassemble the whole product; for a banded pattern that exchange is a halo,
smaller than what the other ranks hold."""

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


def test_owned_ranges_and_exchange_plan():
    for n, r in ((10, 3), (0, 2), (7, 7), (5, 8)):
        rg = shard.owned_ranges(n, r)
        assert len(rg) == r and rg[0][0] == 0 and rg[-1][1] == n
        assert all(x[1] == y[0] for x, y in zip(rg, rg[1:]))
        sizes = [hi - lo for lo, hi in rg]
        assert max(sizes) - min(sizes) <= 1
    rg = [(0, 4), (4, 4), (4, 9), (9, 12)]
    need = np.array([0, 3, 4, 8, 11])
    plan = shard.exchange_plan(need, rg)
    assert sorted(plan) == [0, 2, 3]
    assert np.array_equal(np.concatenate([plan[k] for k in sorted(plan)]), need)
    for k, idx in plan.items():
        assert all(rg[k][0] <= i < rg[k][1] for i in idx)
    assert shard.exchange_plan([], rg) == {}
    with pytest.raises(ValueError):
        shard.exchange_plan([12], rg)
    # pairs of C leaves [1, 3): cseg[1] .. cseg[3] - 1
    cseg = [0, 2, 3, 6]
    pa, pb = [5, 1, 1, 2, 0, 2], [0, 0, 3, 3, 4, 3]
    na, nb = shard.needed_leaves(cseg, pa, pb, 1, 3)
    assert na.tolist() == [0, 1, 2] and nb.tolist() == [3, 4]
    na, nb = shard.needed_leaves(cseg, pa, pb, 2, 2)
    assert na.size == 0 and nb.size == 0


def _morton_plan(a, b):
    """Pairs of a*b from set logic: C leaves in Morton order, each one's pairs
    in ascending K, A and B leaves numbered in their own Morton order."""
    import oracle
    from tests import setref
    oa = np.argsort(oracle.morton_key(a.brow, a.bcol), kind="stable")
    ob = np.argsort(oracle.morton_key(b.brow, b.bcol), kind="stable")
    ia = {(int(a.brow[i]), int(a.bcol[i])): p for p, i in enumerate(oa)}
    ib = {(int(b.brow[i]), int(b.bcol[i])): p for p, i in enumerate(ob)}
    segs = setref.pairs_per_c_leaf(setref.pattern_set(a.brow, a.bcol),
                                   setref.pattern_set(b.brow, b.bcol))
    keys = sorted(segs, key=lambda ij: int(oracle.morton_key([ij[0]], [ij[1]])[0]))
    cseg, pa, pb = [0], [], []
    for I, J in keys:
        for K in segs[(I, J)]:
            pa.append(ia[(I, K)])
            pb.append(ib[(K, J)])
        cseg.append(len(pa))
    return keys, np.array(cseg), np.array(pa), np.array(pb), oa, ob


def _workload(kind):
    import workloads as w
    if kind == "banded":
        return w.config1(1024, 32, 3)
    return (w.random_blocks(1024, 32, 0.12, 21), w.random_blocks(1024, 32, 0.12, 22))


def _rank_main_distributed(rank, world, port, kind, out_q):
    import torch
    import torch.distributed as dist

    import oracle
    import workloads as w
    from paper_2011_11762_gb300 import shard as sh

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = _workload(kind)
        keys, cseg, pa, pb, oa, ob = _morton_plan(a, b)
        bb = a.b * a.b
        # every rank holds one Morton range of each operand at the start
        ra, rb = sh.owned_ranges(oa.size, world), sh.owned_ranges(ob.size, world)
        own_a = {p: a.vals[oa[p]] for p in range(*ra[rank])}
        own_b = {p: b.vals[ob[p]] for p in range(*rb[rank])}
        lo, hi = sh.partition_units(np.diff(cseg), world)[rank]
        need_a, need_b = sh.needed_leaves(cseg, pa, pb, lo, hi)
        plan_a, plan_b = sh.exchange_plan(need_a, ra), sh.exchange_plan(need_b, rb)
        empty = np.zeros(0, dtype=np.int64)
        req = {src: (plan_a.get(src, empty), plan_b.get(src, empty))
               for src in range(world) if src != rank}
        all_req = [None] * world
        dist.all_gather_object(all_req, req)
        ops, keep = [], []
        for dst in range(world):  # serve what dst asked of this rank
            if dst == rank:
                continue
            ia, ib = all_req[dst][rank]
            if ia.size + ib.size == 0:
                continue
            buf = torch.from_numpy(np.concatenate(
                [np.stack([own_a[int(p)] for p in ia]).ravel() if ia.size else np.zeros(0),
                 np.stack([own_b[int(p)] for p in ib]).ravel() if ib.size else np.zeros(0)]))
            keep.append(buf)
            ops.append(dist.isend(buf, dst))
        got = {}
        for src, (ia, ib) in req.items():
            if ia.size + ib.size == 0:
                continue
            buf = torch.empty((ia.size + ib.size) * bb, dtype=torch.float64)
            ops.append(dist.irecv(buf, src))
            got[src] = (ia, ib, buf)
        for op in ops:
            op.wait()
        loc_a = {int(p): own_a[int(p)] for p in need_a if int(p) in own_a}
        loc_b = {int(p): own_b[int(p)] for p in need_b if int(p) in own_b}
        received = 0
        for ia, ib, buf in got.values():
            v = buf.numpy().reshape(-1, a.b, a.b)
            loc_a.update({int(p): v[i] for i, p in enumerate(ia)})
            loc_b.update({int(p): v[ia.size + i] for i, p in enumerate(ib)})
            received += ia.size + ib.size
        assert sorted(loc_a) == need_a.tolist() and sorted(loc_b) == need_b.tolist()

        def local(m, order, loc):
            idx = np.array(sorted(loc), dtype=np.int64)
            src = order[idx]
            vals = np.stack([loc[int(p)] for p in idx]) if idx.size else \
                np.zeros((0, m.b, m.b))
            return oracle.OMatrix.from_block_matrix(
                w.BlockMatrix(m.n, m.b, m.brow[src], m.bcol[src], vals))

        LA, LB = local(a, oa, loc_a), local(b, ob, loc_b)
        mine = {}
        for I, J in keys[lo:hi]:
            v, present = oracle.leaf_product(LA, LB, I, J)
            assert present
            mine[(I, J)] = v
        others = (oa.size - (ra[rank][1] - ra[rank][0])) + (ob.size - (rb[rank][1] - rb[rank][0]))
        gathered = [None] * world
        dist.all_gather_object(gathered, (mine, received, others))
        if rank == 0:
            full = {}
            for part, _, _ in gathered:
                assert not (set(part) & set(full))
                full.update(part)
            FA, FB = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
            cr, cc, _ = (FA @ FB).leaves(values=False)
            assert set(full) == set(zip(cr.tolist(), cc.tolist()))
            # against the same single-leaf product (ascending K) on the whole
            # operands: equal bit for bit
            exact = all(np.array_equal(full[(int(r), int(c))],
                                       oracle.leaf_product(FA, FB, int(r), int(c))[0])
                        for r, c in zip(cr, cc))
            out_q.put(("ok", exact, [(g[1], g[2]) for g in gathered]))
    except Exception as e:  # report to the parent
        out_q.put(("error", repr(e)))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,world", [("banded", 2), ("banded", 3), ("random", 3)])
def test_distributed_operands_exchange_only_needed_leaves(kind, world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main_distributed, args=(r, world, port, kind, q))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = q.get(timeout=10)
    assert res[0] == "ok", res
    _, exact, traffic = res
    assert exact
    if kind == "banded":
        for received, others in traffic:
            assert 0 < received < others / 2, traffic

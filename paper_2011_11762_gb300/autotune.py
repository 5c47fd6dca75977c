"""Leaf-size and schedule autotuner for batched products.

Each product is given once at the finest leaf size (32).  For every product
the tuner builds the candidate blockings (32, and 64 by merging 2 x 2 leaves
with zero fill), runs the symbolic phase for each, times the numeric phase
of each on the GPU and keeps the faster one.  It then times the whole batch
with the longest-first and the Morton work orders and keeps the faster.
Decisions are cached in a JSON file keyed by a hash of each product's
pattern, so a repeated workload is not re-timed.

Reblocking runs on the GPU with torch tensor ops (data preparation, not part
of the product).
"""

from __future__ import annotations

import hashlib
import json
import os

import torch

from . import (CHT_FP64, OPT_SCHEDULE, Batch, cht_mat_from_blocks, cht_multiply,
               cht_symbolic_multiply, get_option, set_option)

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "cht", "autotune.json")


def reblock(n: int, b: int, brow, bcol, vals, b_new: int, device="cuda"):
    """The same matrix with leaf size b_new (a multiple of b dividing n):
    (brow, bcol, vals) of the merged leaves, zero-filled, on ``device``
    (the GPU for the tuner), in row-major order of the new leaves."""
    if b_new == b:
        return brow, bcol, vals
    if b_new % b or n % b_new:
        raise ValueError("b_new must be a multiple of b and divide n")
    f = b_new // b
    g_new = n // b_new
    brow = torch.as_tensor(brow, device=device).long()
    bcol = torch.as_tensor(bcol, device=device).long()
    vals = torch.as_tensor(vals, device=device, dtype=torch.float64)
    key = (brow // f) * g_new + (bcol // f)
    uniq, inv = torch.unique(key, return_inverse=True)
    out = torch.zeros((uniq.numel(), f, b, f, b), dtype=torch.float64, device=device)
    out[inv, brow % f, :, bcol % f, :] = vals
    return ((uniq // g_new).to(torch.int32), (uniq % g_new).to(torch.int32),
            out.reshape(uniq.numel(), b_new, b_new))


def _signature(n, a, bm, mode) -> str:
    h = hashlib.sha1()
    h.update(f"{n}:{mode}:".encode())
    for m in (a, bm):
        for t in (m[0], m[1]):
            h.update(torch.as_tensor(t).to(torch.int32).cpu().numpy().tobytes())
    return h.hexdigest()


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, cache):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, path)
    except OSError:
        pass


class TunedBatch:
    """The tuned batch plus what was chosen."""

    def __init__(self, batch, mats, plans, leaf_sizes, schedule, timings):
        self.batch = batch
        self.mats = mats          # [(A, B)] at the chosen leaf sizes
        self.plans = plans
        self.leaf_sizes = leaf_sizes
        self.schedule = schedule  # "longest-first" or "morton"
        self.timings = timings

    @property
    def useful_flops(self) -> int:
        return self.batch.useful_flops


def tune(products, mode: int = CHT_FP64, candidates=(32, 64), reps: int = 2,
         cache_path: str | None = DEFAULT_CACHE) -> TunedBatch:
    """Tune and build a batch.  ``products`` is a list of (n, (brow, bcol,
    vals) of A, (brow, bcol, vals) of B) at leaf size 32."""
    cache = _load_cache(cache_path) if cache_path else {}
    old_sched = get_option(OPT_SCHEDULE)
    chosen_mats, chosen_plans, sizes, timings = [], [], [], []
    try:
        set_option(OPT_SCHEDULE, 0)
        for n, a, bm in products:
            sig = _signature(n, a, bm, mode)
            cand = [c for c in candidates if n % c == 0]
            best = cache.get(sig)
            options = {}
            for c in ([best] if best in cand else cand):
                A = cht_mat_from_blocks(n, c, *reblock(n, 32, *a, c))
                B = cht_mat_from_blocks(n, c, *reblock(n, 32, *bm, c))
                plan = cht_symbolic_multiply(A, B)
                t = None
                if best not in cand:
                    out, _ = cht_multiply(plan, A, B, mode=mode)
                    t = _time(lambda: cht_multiply(plan, A, B, mode=mode, out=out), reps)
                options[c] = (A, B, plan, t)
            if best not in cand:
                best = min(options, key=lambda c: options[c][3])
                cache[sig] = best
            A, B, plan, t = options[best]
            chosen_mats.append((A, B))
            chosen_plans.append(plan)
            sizes.append(best)
            timings.append({c: options[c][3] for c in options})
        # work order of the whole batch
        best_sched, best_t, best_batch = None, None, None
        for sched, name in ((0, "longest-first"), (1, "morton")):
            set_option(OPT_SCHEDULE, sched)
            bt = Batch(chosen_plans, [m[0] for m in chosen_mats], [m[1] for m in chosen_mats],
                       mode=mode)
            t = _time(bt.run, reps)
            if best_t is None or t < best_t:
                best_sched, best_t, best_batch = name, t, bt
    finally:
        set_option(OPT_SCHEDULE, old_sched)
    if cache_path:
        _save_cache(cache_path, cache)
    return TunedBatch(best_batch, chosen_mats, chosen_plans, sizes, best_sched,
                      {"per_product_ms": timings, "batch_ms": best_t})

"""Host-side logic for running the product on several GPUs (one process per
GPU, torch.distributed).

The product partitions by C leaf: every C leaf is computed from A's leaf row
and B's leaf column alone, and exactly one rank owns it, so no reduction is
needed.  ``partition_units`` cuts the Morton-ordered C leaves into contiguous
ranges of about equal pair count (contiguous Morton ranges keep each rank's
A rows and B columns local, the locality the paper's runtime exploits).
When the operands start distributed (rank r holding a contiguous Morton
range of each operand's leaves, ``owned_ranges``), the only exchange is
one-sided and happens before any arithmetic: a rank needs the A and B leaves
that its C leaves' pairs use (``needed_leaves``), asks each owner for its
share of them (``exchange_plan``) and receives exactly those.  For banded
and 3D-locality patterns that is a halo of neighbouring leaves, not the
whole operand.
The benchmark's multi-GPU mode runs replicas instead (weak scaling, no
collective on the data path); the helpers below also serve its timing
(slowest rank) and totals.
"""

from __future__ import annotations

import numpy as np


def partition_units(seg_lengths, nranks: int):
    """Contiguous [lo, hi) ranges of units, one per rank, splitting the total
    pair count as evenly as contiguity allows (each boundary at the first
    unit whose prefix sum reaches rank * total / nranks)."""
    lens = np.asarray(seg_lengths, dtype=np.int64)
    if nranks <= 0:
        raise ValueError("nranks must be positive")
    n = lens.shape[0]
    prefix = np.concatenate([[0], np.cumsum(lens)])
    total = int(prefix[-1])
    bounds = [0]
    for r in range(1, nranks):
        target = total * r / nranks
        cut = int(np.searchsorted(prefix, target, side="left"))
        bounds.append(min(max(cut, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(nranks)]


def owned_ranges(nleaves: int, nranks: int):
    """Contiguous [lo, hi) ranges of an operand's Morton-ordered leaves, one
    per rank, sizes differing by at most one: the initial distribution."""
    if nranks <= 0:
        raise ValueError("nranks must be positive")
    base, extra = divmod(int(nleaves), nranks)
    out, lo = [], 0
    for r in range(nranks):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def needed_leaves(cseg, pair_a, pair_b, lo: int, hi: int):
    """Sorted distinct A-leaf and B-leaf indices (Morton order) used by the
    pairs of the C leaves [lo, hi): pairs cseg[lo] .. cseg[hi] - 1."""
    cseg = np.asarray(cseg, dtype=np.int64)
    s, e = int(cseg[lo]), int(cseg[hi])
    return (np.unique(np.asarray(pair_a)[s:e]).astype(np.int64),
            np.unique(np.asarray(pair_b)[s:e]).astype(np.int64))


def exchange_plan(needed, ranges):
    """Split sorted leaf indices by owning rank: {rank: indices owned by it},
    ranks with nothing to send left out."""
    needed = np.asarray(needed, dtype=np.int64)
    starts = np.array([lo for lo, _ in ranges], dtype=np.int64)
    ends = np.array([hi for _, hi in ranges], dtype=np.int64)
    if needed.size and (needed[0] < starts.min() or needed[-1] >= ends.max()):
        raise ValueError("leaf index outside every range")
    owner = np.searchsorted(ends, needed, side="right")
    return {int(r): needed[owner == r] for r in np.unique(owner)}


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over all ranks (1 rank: x)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    """Sum of x over all ranks (1 rank: x)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

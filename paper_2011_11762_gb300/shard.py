"""Host-side logic for running the product on several GPUs (one process per
GPU, torch.distributed).

The product partitions by C leaf: every C leaf is computed from A's leaf row
and B's leaf column alone, and exactly one rank owns it, so no reduction is
needed.  ``partition_units`` cuts the Morton-ordered C leaves into contiguous
ranges of about equal pair count (contiguous Morton ranges keep each rank's
A rows and B columns local, the locality the paper's runtime exploits).
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

"""Host logic of multi-GPU runs: one process per GPU, each advancing its own
independent fits, with no collective on the data path.

The M2M workloads partition into independent fits. One fit per GPU (each rank its
own seeded model) gives weak scaling; a batch of fits is split over the ranks by
particle count (largest first to the least-loaded rank) for strong scaling. The
only collective is the reduction of timings to their maximum over ranks.
"""
from __future__ import annotations


def rank_seed(rank: int) -> int:
    """Seed of the initial model of the fit rank `rank` runs alone."""
    return rank


def split_fits(counts, world: int) -> list:
    """Indices of the fits each of `world` ranks runs: longest-processing-time
    assignment by particle count, deterministic (ties go to the lower rank and the
    lower fit index); every fit appears on exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(counts)), key=lambda i: (-int(counts[i]), i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(counts[i])
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the value
    itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])

"""Host logic of multi-GPU runs: one process per GPU.

Independent fits partition with no collective on the data path: one fit per GPU (each
rank its own seeded model) gives weak scaling, and a batch of fits is split over the
ranks by particle count (largest first to the least-loaded rank) for strong scaling.

One fit can also be split over the ranks by particles (the library's shards): each rank
holds a contiguous range, makes the per-particle pass of a step, and the ranks add their
int64 fixed-point sums (one all-reduce per step, NCCL on GPUs) before every rank runs the
same finalize. Integer addition is exact, so the split fit is bit-identical to the whole
one on a single GPU.
"""
from __future__ import annotations

import numpy as np


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


def shard_range(n: int, rank: int, world: int):
    """[lo, hi) of the contiguous particle range rank `rank` of `world` holds: the ranges
    tile [0, n) in rank order and differ in length by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return n * rank // world, n * (rank + 1) // world


def take_range(p: dict, lo: int, hi: int) -> dict:
    """The particles [lo, hi) of a particle dict (copies, contiguous)."""
    return {k: np.ascontiguousarray(v[lo:hi]) for k, v in p.items()}


class ShardDriver:
    """Runs one shard of a split fit through the library's protocol: bounds summed and
    maximised over the ranks, load, then per step begin / exchange / end. `exchange(fit)`
    replaces the shard's exchange words by their sum over the ranks (an all-reduce), and
    `reduce(values, op)` combines host floats over the ranks ("sum" or "max")."""

    def __init__(self, fit, exchange, reduce):
        self.fit = fit
        self.exchange = exchange
        self.reduce = reduce

    def load(self, particles: dict, n_total: int):
        w_sum, v2 = self.fit.shard_bounds(particles)
        w_total = self.reduce(w_sum, "sum")
        v2_bound = self.reduce(v2, "max")
        self.fit.shard_set(n_total, w_total, v2_bound)
        self.fit.load(particles)
        self.exchange(self.fit)
        self.fit.step_end()

    def step(self, k: int = 1):
        for _ in range(k):
            self.fit.step_begin()
            self.exchange(self.fit)
            self.fit.step_end()

    def weights(self):
        self.fit.shard_weights_begin()
        self.exchange(self.fit)
        return self.fit.weights()


def torch_reduce(value: float, op: str) -> float:
    """Sum or maximum of a host float over the default process group (the value itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t[0])


class _DeviceWords:
    """A device int64 array seen through the CUDA array interface (no copy)."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<i8", "data": (ptr, False),
                                         "version": 3, "strides": None}


def nccl_exchange(fit):
    """The shard's exchange words summed over the ranks in place (NCCL all-reduce of int64),
    ordered after the shard's stream work by a synchronisation."""
    import torch
    import torch.distributed as dist
    ptr, count = fit.shard_exchange()
    fit.synchronize()
    words = torch.as_tensor(_DeviceWords(ptr, count), device="cuda")
    dist.all_reduce(words, op=dist.ReduceOp.SUM)
    torch.cuda.current_stream().synchronize()

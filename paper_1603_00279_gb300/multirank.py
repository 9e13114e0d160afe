"""Independent instances over ranks (one process per GPU), host side only.

The time march of one instance is sequential and a single instance does not shard (every FFT
pass would need an all-to-all and every CGS iteration global dot products), so several GPUs only
ever work on different instances: replicas of a single-instance workload, or shards of a set of
independent instances (the batched and history workloads).  No data-path collective exists; the
only cross-rank operation is the reduction of the timing (the slowest rank sets the time).

Shards are balanced by the cost estimate n * M * (I log2 L + M / 2): I CGS iterations of FFT
Toeplitz products of length L per level, plus the history sum that reads M / 2 earlier levels
on average.
"""
from __future__ import annotations

import math
from typing import List, Sequence


def instance_cost(n: int, M: int, iters: float = 10.0) -> float:
    """Estimated work of one instance's march (arbitrary units, comparable across instances)."""
    L = max(8, 1 << math.ceil(math.log2(2 * n)))
    return float(n) * M * (iters * math.log2(L) + M / 2.0)


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time-first assignment of instances to `world` ranks: instances in
    decreasing cost, each to the currently least-loaded rank (ties: lowest rank).  Deterministic,
    so every rank computes the same partition without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def shard(costs: Sequence[float], world: int, rank: int) -> List[int]:
    """Indices of the instances rank `rank` marches."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return partition(costs, world)[rank]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks of the default process group (the value itself when
    no group is initialised): the timing of a step is that of its slowest rank."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

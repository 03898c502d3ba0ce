"""Sharding of independent solves over ranks (one process per GPU, no data-path collective).

The batched sweep's problems are independent eigenproblems of uneven sizes, so a multi-GPU
run partitions them: longest processing time first (largest DOF to the least loaded rank,
ties to the lower rank), which keeps every rank's load within one problem of the mean. Each
rank solves its share with its own iwf_batch_solve; only the timings and the per-problem
results meet on the host afterwards.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition(costs, world: int) -> list[list[int]]:
    """Indices of the problems of every rank, each list ascending. costs: one non-negative
    number per problem (its DOF, say); world >= 1."""
    costs = np.asarray(costs, dtype=np.float64).ravel()
    if world < 1:
        raise ValueError("world must be >= 1")
    if np.any(costs < 0) or not np.all(np.isfinite(costs)):
        raise ValueError("costs must be finite and >= 0")
    order = sorted(range(costs.size), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(v) for v in out]


def shard(costs, world: int, rank: int) -> list[int]:
    """This rank's problems under partition()."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return partition(costs, world)[rank]


def loads(costs, parts) -> np.ndarray:
    costs = np.asarray(costs, dtype=np.float64).ravel()
    return np.array([costs[p].sum() if len(p) else 0.0 for p in parts])

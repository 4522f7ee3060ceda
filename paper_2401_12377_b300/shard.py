"""Splitting the batched and serving workloads over GPUs, and gathering their logs.

One stream has one window and one dependency chain, so it does not shard: a
single stream runs as replicas. The batched and serving workloads are made of
independent streams, so they shard with no data exchange at all: every rank
runs its share of the streams in one persistent launch of its own, and the
host gathers statistics and latency logs afterwards (the only collective).

* ``partition_by_size``: longest-processing-time-first assignment of a batch's
  streams (sorted by task count, each to the rank with the fewest tasks so
  far, ties to the lower rank), so the ranks' makespans stay close.
* ``partition_round_robin``: request i to rank i mod world, which splits a
  Poisson arrival process into world Poisson processes of rate / world.
* ``gather_values`` / ``percentiles``: per-request latencies of every rank
  concatenated on rank 0 in rank order; p50 / p99 over the concatenation, the
  same nearest-rank rule bench.py uses on one GPU.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence, Tuple

import numpy as np


def partition_by_size(sizes: Sequence[int], world: int, rank: int) -> List[int]:
    """Indices (ascending) of the streams rank `rank` of `world` runs: streams
    taken longest first, each to the rank with the least work so far."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    heap = [(0, r) for r in range(world)]
    mine = []
    for i in sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i)):
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return sorted(mine)


def partition_round_robin(n: int, world: int, rank: int) -> np.ndarray:
    """Indices rank, rank + world, ... of n items."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return np.arange(rank, n, world)


def gather_values(dist, values: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Every rank's 1-D float64 array, concatenated in rank order on rank 0
    (other ranks get an empty array). Without a process group: the array."""
    values = np.asarray(values, np.float64)
    if dist is None or world == 1:
        return values
    out = [None] * world if rank == 0 else None
    dist.gather_object(values, out, dst=0)
    return np.concatenate(out) if rank == 0 else np.zeros(0)


def gather_sum(dist, x: float) -> float:
    """The sum of x over all ranks, on every rank (x itself alone)."""
    if dist is None:
        return x
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, float(x))
    return float(sum(out))


def percentiles(values: np.ndarray, ps: Tuple[float, ...] = (0.5, 0.99)) -> List[float]:
    """Nearest-rank percentiles of the sorted values: element min(n - 1, int(p n))."""
    a = np.sort(np.asarray(values, np.float64))
    if not len(a):
        return [float("nan")] * len(ps)
    return [float(a[min(len(a) - 1, int(p * len(a)))]) for p in ps]

"""Sharding of independent systems across ranks (one GPU per rank).

A batch of independent periodic systems has no data-path exchange: each rank
evaluates its own subset and only the timing (max over ranks) is combined.  The
subsets are balanced by an estimated cost per system,

    cost = K^4 + PARTICLE_WEIGHT * n,

the mode products (6 R K^4 flops, R nearly independent of K at a fixed tolerance)
plus the particle work of spreading and gathering (n^3 stencil points per
particle), with the weight taken from measured stage times on one GB300 (K = 64
SKP stages ~170 us, 3e4 particles' spread and gather ~60 us).  The partition is
greedy longest-processing-time first, whose makespan is at most 4/3 of the
optimum (Graham 1969).
"""
from __future__ import annotations

import heapq
from typing import Sequence

PARTICLE_WEIGHT = 200.0


def system_cost(K: int, n: int) -> float:
    """Estimated relative cost of one evaluation of a system with mesh K and n charges."""
    return float(K) ** 4 + PARTICLE_WEIGHT * float(n)


def partition_lpt(costs: Sequence[float], n_ranks: int) -> list[list[int]]:
    """Indices of ``costs`` split into ``n_ranks`` lists by longest processing time first.

    Deterministic (ties broken by index, then by rank), so every rank computes the same
    partition without communicating.  Each list is returned in increasing index order."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(n_ranks)]
    heapq.heapify(heap)
    parts: list[list[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def makespan(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> float:
    return max((sum(float(costs[i]) for i in p) for p in parts), default=0.0)

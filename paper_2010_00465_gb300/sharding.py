"""Splitting independent matrices over ranks (one process per GPU).

Every matrix of a batch is an independent problem, so N ranks need no
collective on the data path: each rank runs the batched path on its own
share.  Shares are balanced by the algorithmic cost of a matrix, taken as
n^3 (the scaling s and family 2m depend on the norm, which is known only on
the device; n^3 is the part known on the host), with the greedy
longest-processing-time rule: matrices in decreasing cost, each to the least
loaded rank so far.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(costs, world: int):
    """Indices of the matrices for every rank (each list in increasing order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def shard(ns, world: int, rank: int):
    """This rank's matrix indices for a batch of orders ``ns``."""
    ns = np.asarray(ns, dtype=np.float64)
    return lpt_partition(ns ** 3, world)[rank]


def imbalance(ns, parts) -> float:
    """Largest rank load over the mean load (1.0 = perfect balance)."""
    ns = np.asarray(ns, dtype=np.float64)
    loads = np.array([float(np.sum(ns[p] ** 3)) for p in parts])
    return float(loads.max() / max(loads.mean(), 1e-300))

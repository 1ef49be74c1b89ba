"""Sharding a batch of independent inversions across ranks (one process per
GPU).  Matrices are independent, so the only exchange is a host-side gather
of results; the data path has no collective.

:func:`partition` assigns matrices to ranks by longest-processing-time first
on the cost n^3: sort by decreasing cost, give each to the rank with the least
load so far (ties to the lowest rank), which keeps the largest load within
4/3 of optimal.
"""
from __future__ import annotations

import heapq


def partition(sizes, world: int) -> list[list[int]]:
    """Indices of `sizes` for each of `world` ranks (each list ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i))
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 3, r))
    return [sorted(p) for p in parts]


def loads(sizes, parts) -> list[int]:
    return [sum(int(sizes[i]) ** 3 for i in p) for p in parts]

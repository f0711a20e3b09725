"""Partition of independent systems over ranks (host logic of the batched workload).

Systems of an uneven batch never interact, so several GPUs take disjoint subsets and
need no collective on the data path.  The estimated cost of a system is its size
(the factorisation is linear in N for a fixed family, Sec. 2.4); longest processing
time first: systems in decreasing cost, each to the currently lightest rank.
"""
from __future__ import annotations

import heapq


def lpt_partition(costs, nranks: int) -> list[list[int]]:
    """Indices of ``costs`` per rank (each list ascending); ties go to the lower rank."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    heap = [(0.0, r) for r in range(nranks)]
    parts = [[] for _ in range(nranks)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]

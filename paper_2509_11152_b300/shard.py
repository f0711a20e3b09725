"""Partition of independent systems over ranks (host logic of the batched workload).

Systems of an uneven batch never interact, so several GPUs take disjoint subsets and
need no collective on the data path.  The estimated cost of a system is its size
(the factorisation is linear in N for a fixed family, Sec. 2.4); longest processing
time first: systems in decreasing cost, each to the currently lightest rank.  Within a
rank, a share larger than the GPU's memory runs as sub-batches (first fit decreasing
on the estimated memory of each system).
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


def memory_bins(costs, capacity: float) -> list[list[int]]:
    """Indices of ``costs`` grouped into sub-batches whose summed cost stays within
    ``capacity`` (first fit in decreasing cost, ties by index; each bin ascending, bins
    in order of creation): the systems a GPU factorises together when its share of a
    batch does not fit in its memory at once.  A single cost above the capacity is a
    ValueError (that system cannot run at all)."""
    if capacity <= 0:
        raise ValueError("capacity must be positive")
    bins: list[list[int]] = []
    loads: list[float] = []
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        c = float(costs[i])
        if c > capacity:
            raise ValueError(f"item {i} of cost {c} exceeds the capacity {capacity}")
        for b, load in enumerate(loads):
            if load + c <= capacity:
                bins[b].append(i)
                loads[b] += c
                break
        else:
            bins.append([i])
            loads.append(c)
    return [sorted(b) for b in bins]

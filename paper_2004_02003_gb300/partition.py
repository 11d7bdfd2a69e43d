"""Assignment of whole blocks to GPUs (host logic, no device code).

BTO advances every block independently for a whole interval (Sec. 3.1), so
a multi-GPU run needs no communication on the data path: each rank takes a
set of whole blocks and advances them in its own batched context. The
blocks are assigned by estimated work (particles times cycles) with the
longest-processing-time rule: blocks in decreasing order of work, each to
the rank with the least work so far (ties to the lowest rank). Every rank
computes the same assignment from the same inputs, so no message is needed
to agree on it.
"""
from __future__ import annotations

import heapq


def block_work(extents, strides, cycles: int = 1):
    """Estimated work of each block: its seed count times the cycles."""
    out = []
    for n, s in zip(extents, strides):
        seeds = 1
        for a in range(3):
            seeds *= -(-int(n[a]) // int(s))
        out.append(seeds * int(cycles))
    return out


def partition_blocks(work, world: int):
    """Blocks of each rank (ascending indices) under the longest-processing-
    time rule; ranks may receive no block when there are fewer blocks than
    ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda b: (-work[b], b))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for b in order:
        load, r = heapq.heappop(heap)
        parts[r].append(b)
        heapq.heappush(heap, (load + work[b], r))
    return [sorted(p) for p in parts]

"""Host-side partitioning for one-process-per-GPU runs.

Fold-in rows are independent given V and batched problems are independent of
one another, so both shard with no exchange on the data path: each rank takes
a contiguous range of rows, or a cost-balanced subset of problems, and keeps
its own copy of V.  Only the timing is reduced across ranks (maximum)."""
from __future__ import annotations

import heapq
from typing import List, Sequence, Tuple


def row_range(m: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous rows [r0, r1) of rank `rank` out of `world`; sizes differ by
    at most one and the ranges tile [0, m) in rank order."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(m), world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Problems to ranks by longest processing time first: problems in
    decreasing cost go to the currently least loaded rank (ties: lower rank).
    Returns, per rank, its problem indices in increasing order."""
    if world <= 0:
        raise ValueError("world must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]

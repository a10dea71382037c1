"""Host-side partitioning for one-process-per-GPU runs.

Fold-in rows are independent given V and batched problems are independent of
one another, so both shard with no exchange on the data path: each rank takes
a contiguous range of rows, or a cost-balanced subset of problems, and keeps
its own copy of V.  Only the timing is reduced across ranks (maximum).

The joint online refit is the one step with a real exchange: V depends on
every row.  With the streaming refit each rank adds its shard's terms to the
per-setting sums of the normal equations; the ranks then sum their
increments (one all-reduce of n x KP x (KP + 1) reals and n counts per batch)
and every rank solves the same V from the same totals."""
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


def allreduce_increments(current, base, group=None):
    """In place: current <- base + the sum over ranks of (current - base).

    `current` are this rank's sums after adding its own shard's terms to the
    common `base` (None: zero); afterwards every rank holds the same totals.
    Works for CPU tensors (gloo) and device tensors (NCCL) alike."""
    import torch.distributed as dist
    for c, b in zip(current, base if base is not None else [None] * len(current)):
        d = c if b is None else c - b
        dist.all_reduce(d, group=group)
        if b is None:
            c.copy_(d)
        else:
            c.copy_(b + d)
    return current


def stream_allreduce(handle, base=None, group=None):
    """Streaming refit across ranks: sum the ranks' increments of the handle's
    per-setting sums since `base` (the totals of the previous exchange, None
    at the start), install the totals and re-solve V.  Returns the new base."""
    sums = list(handle.stream_sums())
    allreduce_increments(sums, base, group)
    handle.stream_set_sums(*sums)
    return [t.clone() for t in sums]

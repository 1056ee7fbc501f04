"""Host-side work split for several GPUs (one process per GPU).

A single inversion does not shard (every block step reads the whole
complement), so single-matrix runs are replicas.  Independent matrices of a
batch or a request stream are split across ranks by estimated cost with no
collective on the data path; only the timing is reduced (max over ranks).
"""
from __future__ import annotations

import heapq


def cost(p: int) -> float:
    """Relative cost of one inversion of order p (every product is O(p^3))."""
    return float(p) ** 3


def shard_by_cost(sizes, world: int, rank: int) -> list:
    """Indices of `sizes` assigned to `rank`: longest-processing-time-first
    greedy over estimated costs (largest matrix to the least loaded rank; ties
    to the lower rank).  Deterministic, so every rank computes the same split
    without communicating."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(sizes)), key=lambda i: (-cost(sizes[i]), i))
    heap = [(0.0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + cost(sizes[i]), r))
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """MAX all-reduce of a scalar over the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

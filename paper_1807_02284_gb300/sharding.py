"""Placement of independent simulations on ranks (one process per GPU).

Batched simulations share nothing, so a multi-GPU run needs no collective on the data path:
each rank advances its own subset.  Subsets are chosen by greedy largest-first bin packing
on the lattice-node count, which keeps the slowest rank (the one that sets the wall time)
close to the mean.  Timing and throughput are combined with one max / sum reduction.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def shard_by_cells(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of `sizes` per rank, largest first onto the least-loaded rank (ties -> lower
    rank).  Every index appears exactly once; each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(s) for s in out]


def rank_share(sizes: Sequence[int], rank: int, world: int) -> List[int]:
    return shard_by_cells(sizes, world)[rank]


def reduce_timing(seconds: float, work: float, group=None):
    """(max seconds over ranks, total work over ranks) with torch.distributed (any backend);
    with no process group the local values are returned."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return seconds, work
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    w = torch.tensor([work], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(w.item())

"""Host-side logic for running the colouring on several GPUs.

Colouring one graph does not shard (it would need a halo exchange every
round), so several GPUs run either independent replicas or disjoint shares
of independent graphs (a batch or a request stream).  There is no collective
on the data path: ranks only agree on the timing at the end.
"""
from __future__ import annotations

import heapq


def shard_graphs(sizes, rank: int, world: int):
    """Indices of the graphs rank `rank` colours: longest-processing-time
    assignment of graphs (by size) to `world` ranks; deterministic, every
    index on exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return sorted(mine)


def aggregate(units: float, seconds: float, group=None, device=None):
    """Whole-job throughput inputs over all ranks: (sum of units, max of
    seconds).  Single process when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(units), float(seconds)
    t = torch.tensor([float(units), float(seconds)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(s.item())

"""Columns across GPUs: the multi-GPU form of the paper's column task queue
(Section 6.2.1, scheme (i)).

Columns (and tables) are independent problems, so ranks exchange no data:
each rank merges the columns assigned to it and only the timing is reduced.
Assignment is longest-processing-time first by the bytes each column's
merge moves (a column's Step 1 + Step 2(b) algorithmic bytes), which
balances the HBM-bound work.
"""
from __future__ import annotations

import heapq

from . import traffic


def column_cost(w: int, m: int, d: int, b: int, n_main: int, n_delta: int) -> int:
    """Bytes a column's merge must move (u bounded by m + d, E'_C by its bound)."""
    u = m + d
    b_new = max(0, (u - 1).bit_length()) if u > 1 else 0
    return traffic.column_bytes(w, m, d, u, b, b_new, n_main, n_delta)


def plan_columns(costs: list[int], world: int) -> list[list[int]]:
    """Column indices per rank: largest first onto the least-loaded rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out: list[list[int]] = [[] for _ in range(world)]
    for idx in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(idx)
        heapq.heappush(heap, (load + costs[idx], r))
    for cols in out:
        cols.sort()
    return out


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_this_rank: int, seconds_this_rank: float, device=None) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    import torch
    import torch.distributed as dist
    units = float(units_this_rank)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        units = float(t.item())
    return units / max_over_ranks(seconds_this_rank, device)

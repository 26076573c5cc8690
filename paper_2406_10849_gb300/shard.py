"""Host-side sharding for multi-GPU runs: independent problems (a batch of
trees, or replicas of one workload) split across ranks with no data-path
exchange.  Only the timing reduction (max over ranks) and the throughput sum use
a collective."""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard_range(num_units: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous, balanced [start, stop) of num_units for this rank."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world")
    base, extra = divmod(num_units, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Greedy longest-processing-time assignment of units (by cost) to ranks."""
    order = sorted(range(len(costs)), key=lambda i: -costs[i])
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    for lst in out:
        lst.sort()
    return out


def shard_problems(problems, rank: int, world: int):
    """This rank's share of a batch of independent tree problems, balanced by
    plan elements per half-step."""
    costs = [float(p.elements_per_half_step()) for p in problems]
    mine = shard_by_cost(costs, world)[rank]
    return [problems[i] for i in mine], mine


def max_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

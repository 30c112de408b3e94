"""Multi-GPU batched runs: independent simulations split across ranks.

Instances of a batch share nothing while they step (each is its own lattice with
its own parameters), so a run on several GPUs needs no exchange until the end:
every rank advances its own shard of the instance list in one context on its
own GPU, and the per-instance results are gathered once. One process per GPU,
torch.distributed for the final gather and the timing reduction only.

The split balances lattice updates: instances are taken largest first and each
goes to the rank with the fewest cells so far (longest-processing-time rule),
ties to the lower rank, so every rank computes the same split from the same
list without communicating.
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def partition(cells: Sequence[int], world: int) -> List[List[int]]:
    """Instance indices per rank (each list ascending), balanced by cell count."""
    if world < 1:
        raise ValueError("world size must be at least 1")
    if any(int(c) < 0 for c in cells):
        raise ValueError("cell counts must be non-negative")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += int(cells[i])
    return [sorted(s) for s in shards]


def shard(cells: Sequence[int], rank: int, world: int) -> List[int]:
    """This rank's instance indices."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return partition(cells, world)[rank]


def imbalance(cells: Sequence[int], world: int) -> float:
    """Largest shard's cells over the mean (1.0 = perfect balance)."""
    loads = [sum(int(cells[i]) for i in s) for s in partition(cells, world)]
    mean = sum(loads) / world
    return max(loads) / mean if mean > 0 else 1.0


def gather_by_instance(local: Dict[int, dict], n_instances: int, group=None) -> List[dict]:
    """All ranks' {instance index: result} merged into one list in instance order
    (on every rank). Raises if an index is missing or claimed twice."""
    import torch.distributed as dist
    parts: List[Dict[int, dict]] = [None] * dist.get_world_size(group)  # type: ignore[list-item]
    dist.all_gather_object(parts, dict(local), group=group)
    merged: Dict[int, dict] = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError("instance %d reported by two ranks" % k)
            merged[int(k)] = v
    missing = [k for k in range(n_instances) if k not in merged]
    if missing or len(merged) != n_instances:
        raise RuntimeError("instances missing from the gather: %s" % missing[:8])
    return [merged[k] for k in range(n_instances)]


def max_over_ranks(value: float, group=None, device=None) -> float:
    """Largest value over the ranks (the whole job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

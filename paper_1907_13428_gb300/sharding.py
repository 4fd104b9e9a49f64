"""Host-side logic of multi-GPU runs: independent instances are sharded across
ranks (one process per GPU) with no data-path collective; the only
communication is the max-over-ranks reduction of the timed region and the
gather of per-instance statistics.

A batch of uneven instances is split by estimated cost (N log N of the
largest axis), greedily: instances in decreasing cost go to the currently
least-loaded rank, ties to the lowest rank, so every rank computes the same
assignment without communicating."""
from __future__ import annotations

import math
from typing import List, Sequence

import torch
import torch.distributed as dist


def instance_cost(nx: int, ny: int, nt: int) -> float:
    """Relative cost of one PCG iteration: transforms of all N points."""
    N = nx * ny * nt
    return N * math.log2(2 * max(nx, ny, nt))


def shard(costs: Sequence[float], world: int) -> List[List[int]]:
    """Instance indices of each rank (longest-processing-time greedy)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_objects(obj):
    """List of every rank's object, in rank order (single-process: [obj])."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out

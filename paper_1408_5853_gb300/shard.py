"""Sharding of independent problem instances over ranks (one GPU per rank).

Instances of a batched sweep share nothing, so a multi-GPU run splits them
across ranks with no exchange on the data path; the only collective is the
max-reduction of the timed region.  Shards are balanced by node count with
the greedy largest-first rule (deterministic: ties go to the lower rank).
"""
from __future__ import annotations


def balanced_shards(sizes: list[int], world: int) -> list[list[int]]:
    """Instance indices per rank, largest instances first onto the least-loaded rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += sizes[k]
    return [sorted(s) for s in out]


def max_over_ranks(x: float, device=None) -> float:
    """Max of a host float over the ranks of the default process group (or x)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Multi-GPU layout of the IoU workloads: independent replicas, no exchange.

Every pair, matrix entry and scene is independent, so N GPUs run N replicas:
each rank takes a contiguous shard of a global pair range (or its own seeded
workload for weak scaling) and the job's time is the slowest rank's.  The only
collectives are the timing barrier and one max-reduction of a scalar; nothing
on the data path is exchanged.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int):
    """Contiguous [start, stop) shard of n units for `rank` of `world`; shards
    cover [0, n) exactly once and differ in size by at most one."""
    if world <= 0 or not (0 <= rank < world) or n < 0:
        raise ValueError(f"bad shard request n={n} rank={rank} world={world}")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def replica_seed(rank: int, base: int = 0) -> int:
    """Seed of rank's own workload in weak-scaling runs."""
    return base + rank


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the job time of a replicated step)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

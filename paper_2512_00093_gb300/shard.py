"""Multi-GPU sharding of the partitioned workload (weak scaling).

Streams are independent units (Sec. 1): rank r of N takes the stream indices
k = r*n .. r*n + n - 1 of the same (seed, J), so every rank jumps and
generates its own disjoint blocks of the one sequence and no data crosses
ranks.  The only collectives are the timing barrier and the max-over-ranks
reduction of the step time.
"""
from __future__ import annotations


def shard(rank: int, world: int, n_per_rank: int) -> tuple[int, int]:
    """(k0, n): the first stream index and the stream count of this rank."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank * n_per_rank, n_per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (the slowest rank sets the step time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

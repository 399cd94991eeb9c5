"""Multi-GPU sharding of the partitioned workload (weak scaling).

Streams are independent units (Sec. 1): stream k of (seed, J) is the block of
the one sequence that starts k*J transitions after the seeded state, so
disjoint index ranges give disjoint blocks and no data crosses ranks.  With N
ranks of n streams each, batch i of rank r is k = (i*N + r)*n .. (i*N + r)*n
+ n - 1: the batches of all ranks and steps tile 0, 1, 2, ... in order, with
no index used twice.  The only collectives are the timing barrier and the
max-over-ranks reduction of the step time.
"""
from __future__ import annotations


def step_k0(step: int, rank: int, world: int, n_per_rank: int) -> int:
    """First stream index of batch `step` on `rank` (each batch n_per_rank
    consecutive streams; batch i of rank r is block i*world + r)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    if step < 0 or n_per_rank < 0:
        raise ValueError("step and n_per_rank must be non-negative")
    return (step * world + rank) * n_per_rank


def shard(rank: int, world: int, n_per_rank: int) -> tuple[int, int]:
    """(k0, n): the first stream index and the stream count of this rank's
    first batch (step 0)."""
    return step_k0(0, rank, world, n_per_rank), n_per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (the slowest rank sets the step time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

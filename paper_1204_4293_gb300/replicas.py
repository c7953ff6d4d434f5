"""Host-side logic for running the pipeline as independent replicas, one
process per GPU (the maps shard across ranks; no data crosses ranks).

Only two things cross ranks: a barrier around the timed region and one
scalar all-reduce (max) of the measured time.  Noise maps can also split
their realisations: each rank adds its range (noise_range) to partial sums
with fm_map_noise_accumulate, merge_noise_sums adds the ranks' sums, and one
rank finalizes them.
"""
from __future__ import annotations

import os


def world_info() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Distinct, reproducible input seeds per rank (maps are independent)."""
    return int(base) + 1000 * (int(rank) + 1)


def shard_maps(total_maps: int, world: int, rank: int) -> range:
    """Contiguous block of map indices owned by `rank` (strong-scaling split)."""
    per, extra = divmod(int(total_maps), int(world))
    start = rank * per + min(rank, extra)
    return range(start, start + per + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a scalar over all ranks (the slowest replica sets the time)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds


def noise_range(total_realisations: int, world: int, rank: int) -> range:
    """The realisations (generator indices) that `rank` accumulates."""
    return shard_maps(total_realisations, world, rank)


def merge_noise_sums(sums):
    """Sum of every rank's partial noise sums, in place (one all-reduce of
    the [2, J-1, n, n] tensor; a no-op on one process)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    return sums

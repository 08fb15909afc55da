"""Host-side logic of multi-GPU runs: one cube per rank (replicas).

The MUFFIN pass shards by channel except for its spectral step, and every box
here has one GPU, so a multi-GPU run solves one independent cube per rank: no
collective touches the data path.  Only the timing crosses ranks (the job's
step time is the slowest rank's) and the throughput adds up.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Each rank solves its own cube: the workload's seed plus the rank."""
    return base_seed + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's step time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, n_ranks: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * n_ranks / seconds

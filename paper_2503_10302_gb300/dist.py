"""Multi-GPU partition of the path (one process per GPU).

The hot path has no exchange step: DT-SQA runs, APT instances and training
instances are independent units.  Ranks therefore take disjoint slices of
the unit range (weak scaling) and the only collectives are the barrier and
the max-over-ranks reduction of the timed region.
"""
from __future__ import annotations

import os
from typing import Tuple


def env_rank() -> Tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def run_ids(step: int, rank: int, world: int, runs_per_rank: int) -> int:
    """First run id of this rank's batch in a given step: batches of all
    ranks and steps are disjoint, so every anneal draws fresh randomness."""
    return (step * world + rank) * runs_per_rank


def shard(n_units: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [begin, end) slice of n_units for this rank (sizes differ by
    at most one)."""
    base, extra = divmod(n_units, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity without a group)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

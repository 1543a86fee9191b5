"""Work division across GPUs (one process per GPU).

The proxy check shards with no exchange: every query is scored independently
against a replicated model, every scene is independent, and Fastron training
is a sequential greedy loop that runs as a replica per scene.  Ranks therefore
share nothing on the data path; the only collective is the max of the step
times, taken so that the reported rate is the whole job's (weak scaling:
each rank does a fixed amount of work).  This module holds that host-side
logic so that it can be tested with the gloo backend on CPU.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return ws, rank, local


def rank_trial(rank: int) -> int:
    """The scene each rank runs: trial = rank, so the seeds differ per rank."""
    return rank


def contiguous_range(n: int, rank: int, ws: int) -> tuple[int, int]:
    """[lo, hi) of n items for this rank, sizes differing by at most one."""
    base, extra = divmod(n, ws)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks (the slowest rank's time); identity
    without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, ws: int, max_ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest time."""
    return ws * units_per_rank / (max_ms * 1e-3)

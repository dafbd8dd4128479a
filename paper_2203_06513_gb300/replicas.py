"""Host logic for runs on several GPUs of one node: ranks, barrier, slowest time.

Two kinds of multi-rank run use it.  Independent replicas (ensembles, and the
default of the measurement): each rank advances its own plasma, drawn from its
own seed, and no data crosses ranks.  One plasma split by markers
(`split.py`): the markers are independent given the fields, so each rank holds
a share of them and every sum over markers (deposits, charge, energies, the
fixed-point test's largest increment) is all-reduced through the library's
reduction callback.  In both, the only collectives added here are the timing
barrier and the max-over-ranks of the timed durations; the whole-job rate is
the units all ranks processed divided by the slowest rank's time (weak scaling:
the work per rank is fixed).
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment; (1, 0, 0) alone."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws < 1 or not 0 <= rank < ws or local < 0:
        raise ValueError(f"bad rank environment: WORLD_SIZE={ws} RANK={rank} LOCAL_RANK={local}")
    return ws, rank, local


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s plasma: distinct per rank, equal to `base` on rank 0."""
    return base + rank


def barrier(ws: int, sync=None) -> None:
    """Finish this rank's device work (`sync`), then wait for every rank."""
    if sync is not None:
        sync()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int, device: str = "cpu") -> float:
    """Largest `v` over all ranks (the slowest rank's time); `v` itself alone."""
    if ws == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, steps: int, seconds: float) -> float:
    """Units all ranks processed per second: ws * units_per_rank * steps / seconds,
    `seconds` being the max over ranks."""
    if seconds <= 0:
        raise ValueError("timed region must have a positive duration")
    return ws * units_per_rank * steps / seconds

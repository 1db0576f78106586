"""Replica bookkeeping for multi-GPU runs.

The local estimator shards into independent configurations with no exchange
step, so N GPUs run N independent replicas.  These helpers reduce per-rank
timings and work counts with torch.distributed (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _reduce(value: float, op, device) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    return _reduce(value, dist.ReduceOp.SUM, device)


def throughput(units_local: float, ms_local: float, device="cpu") -> tuple[float, float]:
    """Whole-job units/s: all ranks' units over the slowest rank's time.
    Returns (units per second, slowest rank's milliseconds)."""
    ms = max_over_ranks(ms_local, device)
    units = sum_over_ranks(units_local, device)
    return units / (ms / 1e3), ms

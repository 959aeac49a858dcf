"""Multi-GPU layout of the benchmark: one independent event (SMC run) per rank.

SMC runs on different events share nothing, so the ranks exchange no data
on the hot path; only two scalars cross ranks per measurement: the summed
evaluation count and the maximum elapsed time (whole-job throughput =
sum of work / slowest rank). Sharding one event's particles across GPUs
would need the per-stage exchange (ESS sums, logsumexp, the integer prefix
offsets of systematic resampling, particle migration), which is not built.
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, world size, local rank) from the torchrun environment (1 process: 0, 1, 0)."""
    g = lambda k, d: int(os.environ.get(k, d))
    return g("RANK", 0), g("WORLD_SIZE", 1), g("LOCAL_RANK", 0)


def event_seed(rank: int) -> int:
    """Seed of the synthetic event analysed by `rank` (each rank: its own injection and noise)."""
    return rank


def run_key(base: int, rank: int, step: int) -> int:
    """Philox key of SMC run `step` on `rank`: disjoint across ranks and steps."""
    return base + 1000 * rank + step


def reduce_scalar(x: float, op: str, world: int, device="cpu") -> float:
    """All-reduce one float across ranks ('sum' or 'max'); identity with one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t[0])


def aggregate(evals: float, seconds: float, world: int, device="cpu"):
    """Whole-job (evaluations/s, slowest rank's seconds)."""
    total = reduce_scalar(evals, "sum", world, device)
    slowest = reduce_scalar(seconds, "max", world, device)
    return total / slowest, slowest

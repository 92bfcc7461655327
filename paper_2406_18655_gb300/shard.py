"""Multi-process data parallelism of the batched decoder (host logic only).

Shots are independent, so N processes (one per GPU) each decode a disjoint range of the
seeded shot stream with no collective on the data path; the only exchanges are the
timing reduction (the job's step time is the slowest rank's) and the sum of per-rank
counts.  Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def shard(rank: int, world: int, shots_per_rank: int) -> tuple[int, int]:
    """(first shot index, shot count) of `rank`: rank r owns shots
    [r * shots_per_rank, (r + 1) * shots_per_rank) of the seeded stream (weak scaling)."""
    if world < 1 or not 0 <= rank < world or shots_per_rank < 0:
        raise ValueError("bad shard request")
    return rank * shots_per_rank, shots_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of `value` over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_per_step_local: float, device=None) -> dict:
    """Whole-job throughput: all ranks' units over the slowest rank's step time."""
    ms = max_over_ranks(ms_per_step_local, device)
    units = sum_over_ranks(units_per_rank, device)
    return {"ms_per_step": ms, "units": units, "per_s": units / (ms / 1000.0)}

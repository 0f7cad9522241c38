"""Replica data parallelism for the exponentiation workloads.

Instances are independent, so N GPUs run N replicas: rank r generates and processes
its own batch (seeded by r), nothing is exchanged on the data path, and the only
collective is the maximum of the timed region over the ranks (the job ends when the
slowest rank ends). One process per GPU; ranks, world size and rendezvous come from
torchrun's environment. This module has no CUDA dependency of its own: the same host
logic runs over gloo on CPU in the tests.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankInfo:
    world: int
    rank: int
    local: int


def rank_info(env=None) -> RankInfo:
    env = os.environ if env is None else env
    return RankInfo(int(env.get("WORLD_SIZE", "1")), int(env.get("RANK", "0")), int(env.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's batch: disjoint synthetic inputs per replica."""
    return base_seed + rank


def init(info: RankInfo, backend: str | None = None):
    """Join the process group when world > 1 (nccl on GPUs, gloo otherwise)."""
    if info.world <= 1:
        return
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))


def barrier(info: RankInfo):
    if info.world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(info: RankInfo, value: float, device=None) -> float:
    """The largest value over all ranks (every rank gets it)."""
    if info.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(info: RankInfo, units_per_rank: int, ms_max: float) -> float:
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    return info.world * units_per_rank / (ms_max / 1e3)

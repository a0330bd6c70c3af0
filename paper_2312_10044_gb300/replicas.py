"""Host coordination of independent replicas of the solve on several GPUs.

The pair passes need no exchange between GPUs when each GPU solves its own
problems (the benchmark runs one replica of the workload per GPU), so the
multi-GPU path is replicas only: one process per GPU, a barrier around the
timed region, and the time taken as the maximum over the processes.  These
helpers hold that logic; they run over NCCL on GPUs and over gloo on CPUs.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def ranks() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> tuple[int, int, int]:
    """Join the process group when there is more than one process."""
    world, rank, local = ranks()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world: int) -> None:
    if world > 1:
        dist.barrier()


def max_over_ranks(x: float, world: int, device: torch.device | str = "cpu") -> float:
    """The largest x over all processes (x itself for one process)."""
    if world <= 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_replica: float, world: int, seconds: float) -> float:
    """Units all replicas processed per second of the slowest replica."""
    return world * units_per_replica / seconds


def finish(world: int) -> None:
    if world > 1 and dist.is_initialized():
        dist.destroy_process_group()

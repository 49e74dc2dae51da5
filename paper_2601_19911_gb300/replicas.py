"""Replica bookkeeping for runs on N GPUs: one process per GPU, each running
the whole workload on its own inputs, with no collective on the data path
(the primitives shard by independent queries, so N GPUs are N replicas).
The launcher (torchrun) sets RANK / LOCAL_RANK / WORLD_SIZE; the timed
region is bracketed by a barrier, the job's time is the maximum over ranks,
and its throughput is all ranks' units over that time."""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's `x` (a time): all ranks get it."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Throughput of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds

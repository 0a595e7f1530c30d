"""Host-side logic of multi-GPU runs: one process per GPU, independent problems.

The method shards into independent units (a DEOCT fit per rank here; MH nodes
of a level and serving jobs likewise), so ranks exchange nothing on the data
path: each rank solves its own problem with its own Philox stream id, and only
the timing is reduced (max over ranks) for the whole-job throughput.
"""
from __future__ import annotations

import os


def env_ranks():
    """(rank, world, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, world: int):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def stream_id(rank: int) -> int:
    """Philox stream id of rank's independent problem."""
    return int(rank)


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time (weak scaling)."""
    return units_per_rank * world / seconds_max

"""Process-group helpers for running independent solves on several GPUs.

Each rank solves its own problem (the space-time solve needs no data
exchange between ranks in this configuration); the only collectives are a
barrier around the timed region and a MAX reduction of the elapsed time, so
that the whole-job throughput is (units processed by all ranks) / (slowest
rank's time).
"""
import os

import torch
import torch.distributed as dist


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, device=None):
    rank, world, local = env()
    if world > 1 and not dist.is_initialized():
        kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
        dist.init_process_group(backend, **kw)
    return rank, world, local


def barrier():
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x, device="cpu"):
    """Maximum of a float over all ranks (x itself without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, max_seconds):
    """Whole-job rate: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / max_seconds


def finalize():
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()

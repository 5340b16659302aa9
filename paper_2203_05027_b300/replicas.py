"""Replica runs on several GPUs of one node: one process per GPU, each solving its own seeded
instance, with no collective on the data path. The only exchanges are the timing ones below
(a barrier around the timed region and the maximum of the per-rank times)."""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest `value` over all ranks of the initialised process group (the job's time is the
    slowest rank's); `value` itself without a group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)

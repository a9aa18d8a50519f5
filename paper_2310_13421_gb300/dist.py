"""Host-side logic of multi-GPU runs: one process per GPU, each decomposing its
own matrices (independent problems: no exchange between ranks on the data
path, so no collective beyond the timing barrier and the max-over-ranks
reduction).  Works with any torch.distributed backend (NCCL on GPUs, gloo on
the CPU for tests)."""
import os

import torch


def rank_env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank, world):
    """Round-robin share of a batch for one rank: item i goes to rank i % world."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %d of %d" % (rank, world))
    return [x for i, x in enumerate(items) if i % world == rank]


def max_over_ranks(x, group=None, device="cpu"):
    """Largest value of x over the ranks (x itself without torch.distributed)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(x, group=None, device="cpu"):
    """Sum of x over the ranks (x itself without torch.distributed)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def job_rate(units_all_ranks, slowest_ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    if slowest_ms <= 0:
        raise ValueError("non-positive time")
    return units_all_ranks / (slowest_ms * 1e-3)

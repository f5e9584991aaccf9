"""Multi-process helpers for running one population per GPU (weak scaling).

Populations on different ranks are independent, so the hot path exchanges
nothing; the only collectives are the timing barrier and the max over ranks
of the step time that bench.py reports.  Works with the nccl backend (one
rank per GPU) and with gloo (CPU tests).
"""
from __future__ import annotations

import os


def world_info():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value of x over all ranks (x itself on one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(units, world, rank):
    """Contiguous share [begin, end) of `units` for `rank` (sizes differ by at most 1)."""
    base, extra = divmod(units, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def weak_scaling_value(units_per_rank, step_seconds, world):
    """Whole-job throughput: units processed on all ranks / the slowest rank's time."""
    total = sum_over_ranks(units_per_rank, world)
    return total / max_over_ranks(step_seconds, world)

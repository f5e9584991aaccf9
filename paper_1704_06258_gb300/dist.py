"""Multi-process helpers: one population per GPU (weak scaling) and one
island population sharded over GPUs (§5 islands, merged across GPUs).

Independent populations exchange nothing on the hot path; the only
collectives are the timing barrier and the max over ranks of the step time
that bench.py reports.  A sharded population exchanges at every island
merge (every N1 generations, §5 outer loop): an all-reduce-min over the
packed key (ancestor fitness, global island index) finds the best island,
and its owner broadcasts the winning n-bit hub mask (nw 32-bit words).  The
library draws the shards' random numbers by global chromosome index, so the
sharded run makes the decisions one GPU holding every island makes.  Works
with the nccl backend (one rank per GPU, tensors on the GPU) and with gloo
(CPU tests).
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


def pack_key(fit, island):
    """64-bit key ordered like (fitness, global island index) for fitness >= 0:
    the IEEE-754 bits of a non-negative float32 sort like its value; a NaN
    fitness ranks after every number (as +inf)."""
    import numpy as np
    f = np.float32(fit)
    if np.isnan(f):
        f = np.float32(np.inf)
    bits = int(np.array([abs(f)], dtype=np.float32).view(np.uint32)[0])
    return (bits << 32) | int(island)


def unpack_key(key):
    import numpy as np
    return float(np.array([key >> 32], dtype=np.uint32).view(np.float32)[0]), int(key & 0xFFFFFFFF)


def exchange_best(fit, island, mask, islands_per_rank, world):
    """The cross-GPU merge step: every rank offers its best island (fitness,
    global index, hub mask as uint32 words); returns the winner's (fitness,
    global island, mask) on every rank.  Ties go to the lowest global island."""
    import numpy as np
    if world == 1:
        return float(fit), int(island), np.asarray(mask, dtype=np.uint32).copy()
    import torch
    import torch.distributed as dist
    dev = _device()
    key = torch.tensor([pack_key(fit, island)], dtype=torch.int64, device=dev)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    wfit, wisland = unpack_key(int(key.item()))
    buf = torch.from_numpy(np.asarray(mask, dtype=np.uint32).view(np.int32).copy()).to(dev)
    dist.broadcast(buf, src=wisland // islands_per_rank)
    return wfit, wisland, buf.cpu().numpy().view(np.uint32).copy()


def sharded_solve(gi, generations, seed, islands_per_rank, island_size, n1, rank, world, stream=0,
                  on_generation=None, on_merge=None):
    """One island population of world * islands_per_rank islands, this rank
    holding islands [rank * islands_per_rank, (rank + 1) * islands_per_rank)
    of it on its GPU (an Instance).  The library runs the generations with its
    own merge turned off (each replayed from its CUDA graph); after every n1
    generations the ranks merge through exchange_best.  Returns the global
    best (hubs, S, cost_fp64, cost_fp32) on every rank; between ranks, equal
    best fitness goes to the lower rank.

    Observers (optional, for checks and tracing): on_generation(g, gi) after
    generation g has run on this rank, before any merge; on_merge(g, wfit,
    wisland, wmask) after the merge that follows generation g."""
    import numpy as np
    gi.set_params(islands=islands_per_rank, island_size=island_size, n1=0,
                  island_offset=rank * islands_per_rank)
    gi.ga_begin(seed, stream)
    for g in range(generations):
        gi.ga_run(1, stream)
        if on_generation is not None:
            on_generation(g, gi)
        if n1 > 0 and (g + 1) % n1 == 0:
            masks, fit = gi.ga_islands(stream)
            key = np.where(np.isnan(fit), np.inf, fit)
            r = int(np.argmin(key))
            wfit, wisland, wmask = exchange_best(fit[r], rank * islands_per_rank + r, masks[r], islands_per_rank,
                                                 world)
            gi.ga_merge(wmask, wfit, stream)
            if on_merge is not None:
                on_merge(g, wfit, wisland, wmask)
    res = gi.ga_result(stream)
    return best_over_ranks(res, rank, world)


def best_over_ranks(res, rank, world):
    """The result with the smallest fp32 fitness over ranks (lowest rank on ties)."""
    if world == 1:
        return res
    import numpy as np
    import torch
    import torch.distributed as dist
    dev = _device()
    key = torch.tensor([pack_key(res["cost_fp32"], rank)], dtype=torch.int64, device=dev)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    _, src = unpack_key(int(key.item()))
    hubs = torch.from_numpy(np.asarray(res["hubs"], dtype=np.int32).copy()).to(dev)
    S = torch.from_numpy(np.asarray(res["S"], dtype=np.int32).copy()).to(dev)
    cost = torch.tensor([res["cost_fp64"], res["cost_fp32"]], dtype=torch.float64, device=dev)
    for t in (hubs, S, cost):
        dist.broadcast(t, src=src)
    c = cost.cpu().numpy()
    return {"hubs": hubs.cpu().numpy(), "S": S.cpu().numpy(), "cost_fp64": float(c[0]),
            "cost_fp32": float(c[1]), "rank": src}

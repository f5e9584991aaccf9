"""Multi-rank helpers on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1704_06258_gb300 import dist as pdist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = pdist.world_info()
        pdist.barrier(w)
        mx = pdist.max_over_ranks(1.5 + rank, w)
        v = pdist.weak_scaling_value(4096, 0.5 + 0.25 * rank, w)
        b, e = pdist.shard(10, w, r)
        q.put((rank, w, r, lr, mx, v, b, e))
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, (r0, w, r, lr, mx, v, b, e) in enumerate(out):
        assert (r0, w, r, lr) == (rank, 2, rank, rank)
        assert mx == 2.5                      # max over ranks
        assert v == pytest.approx(8192 / 0.75)  # all ranks' units / slowest rank
    assert [(o[6], o[7]) for o in out] == [(0, 5), (5, 10)]


def test_shard_covers_everything_once():
    for units in (0, 1, 7, 64, 1000):
        for world in (1, 2, 3, 8):
            spans = [pdist.shard(units, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == units
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1


def _exchange_worker(rank, world, port, q):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        masks = [np.array([0x5, 0x1], np.uint32), np.array([0xA, 0x2], np.uint32)]
        out = []
        # (fitness offered by rank 0, by rank 1): rank 1 wins, tie -> lower island, NaN loses
        for f0, f1 in ((2.0, 1.0), (1.0, 1.0), (float("nan"), 5.0)):
            fit = f0 if rank == 0 else f1
            island = 1 if rank == 0 else 3          # two islands per rank, global ids 0..3
            wf, wi, wm = pdist.exchange_best(fit, island, masks[rank], 2, world)
            out.append((wf, wi, wm.tolist()))
        res = {"hubs": np.array([rank, 9]), "S": np.array([rank] * 4), "cost_fp64": 10.0 - rank,
               "cost_fp32": 10.0 - rank}
        best = pdist.best_over_ranks(res, rank, world)
        out.append((best["rank"], best["cost_fp64"], best["hubs"].tolist()))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_cross_rank_island_merge_on_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_exchange_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    outs = dict(q.get(timeout=10) for _ in range(world))
    assert outs[0] == outs[1]
    o = outs[0]
    assert o[0] == (1.0, 3, [0xA, 0x2])
    assert o[1] == (1.0, 1, [0x5, 0x1])
    assert o[2] == (5.0, 3, [0xA, 0x2])
    assert o[3] == (1, 9.0, [1, 9])


def test_pack_key_orders_fitness_then_island():
    import numpy as np
    pairs = [(0.0, 7), (1.5, 2), (1.5, 3), (1e30, 0), (float("inf"), 0), (float("nan"), 1)]
    keys = [pdist.pack_key(f, i) for f, i in pairs]
    assert keys == sorted(keys)
    assert pdist.unpack_key(keys[1]) == (1.5, 2)
    assert np.isinf(pdist.unpack_key(keys[-1])[0])

"""One rank of a sharded island population (spawned by tests/test_gpu_shards.py).

Each rank runs dist.sharded_solve on its own share of the islands, on cuda:0,
exchanging through a gloo process group, and records what the test compares:
every generation's children and fitness and the ancestors after selection,
every merge's winner and the ancestors after it, and the final result."""
import os
import sys


def run(rank, world, port, out_dir, case):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch
    import torch.distributed as tdist

    from paper_1704_06258_gb300 import dist, synth
    from paper_1704_06258_gb300.binding import Instance

    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        inst = synth.clustered(seed=case["inst_seed"], n=case["n"], p=case["p"])
        gens, merges = [], []
        with Instance.from_instance(inst) as gi:
            gi.set_params(path=case["path"])

            def on_generation(g, h):
                masks, fit = h.ga_population()
                anc, af = h.ga_islands()
                gens.append((masks, fit, anc, af))

            def on_merge(g, wfit, wisland, wmask):
                anc, af = gi.ga_islands()
                merges.append((g, np.float32(wfit), wisland, np.asarray(wmask, dtype=np.uint32), anc, af))

            res = dist.sharded_solve(gi, case["G"], case["seed"], case["R"], case["P"], case["N1"], rank, world,
                                     on_generation=on_generation, on_merge=on_merge)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"),
                 children=np.stack([x[0] for x in gens]), fit=np.stack([x[1] for x in gens]),
                 anc=np.stack([x[2] for x in gens]), anc_fit=np.stack([x[3] for x in gens]),
                 merge_g=np.array([m[0] for m in merges], dtype=np.int64),
                 merge_fit=np.array([m[1] for m in merges], dtype=np.float32),
                 merge_island=np.array([m[2] for m in merges], dtype=np.int64),
                 merge_mask=np.stack([m[3] for m in merges]) if merges else np.zeros((0, 1), np.uint32),
                 merge_anc=np.stack([m[4] for m in merges]) if merges else np.zeros((0, 1, 1), np.uint32),
                 merge_anc_fit=np.stack([m[5] for m in merges]) if merges else np.zeros((0, 1), np.float32),
                 hubs=np.asarray(res["hubs"]), S=np.asarray(res["S"]),
                 cost=np.array([res["cost_fp64"], res["cost_fp32"]]), src=np.array([res["rank"]]))
    finally:
        tdist.destroy_process_group()

"""An island population split over two library handles (the per-GPU shards of
a multi-GPU run, here both on one GPU and merged on the host between
generations) against one handle holding every island."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance, UsaphmpError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def host_merge(shards, per):
    """The cross-shard merge: best ancestor over all islands (NaN last, lowest
    global island on ties) into every island of every shard."""
    best = None
    for k, gi in enumerate(shards):
        masks, fit = gi.ga_islands()
        key = np.where(np.isnan(fit), np.inf, fit)
        r = int(np.argmin(key))
        if best is None or key[r] < best[0]:
            best = (key[r], masks[r].copy(), fit[r])
    for gi in shards:
        gi.ga_merge(best[1], best[2])


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_two_shards_follow_the_whole_population(path):
    inst = synth.urand200(seed=57, n=180, p=7)
    seed, P, N1, blocks = 31, 16, 4, 5
    with Instance.from_instance(inst) as whole, Instance.from_instance(inst) as s0, \
            Instance.from_instance(inst) as s1:
        whole.set_params(islands=6, island_size=P, n1=N1, path=path)
        s0.set_params(islands=3, island_size=P, n1=0, island_offset=0, path=path)
        s1.set_params(islands=3, island_size=P, n1=0, island_offset=3, path=path)
        for gi in (whole, s0, s1):
            gi.ga_begin(seed)
        for _ in range(blocks):
            for gi in (whole, s0, s1):
                gi.ga_run(N1)
            host_merge([s0, s1], 3)
            wm, wf = whole.ga_islands()
            m0, f0 = s0.ga_islands()
            m1, f1 = s1.ga_islands()
            np.testing.assert_array_equal(np.concatenate([m0, m1]), wm)
            np.testing.assert_array_equal(np.concatenate([f0, f1]), wf)
        rw, r0, r1 = whole.ga_result(), s0.ga_result(), s1.ga_result()
    best = r0 if r0["cost_fp32"] <= r1["cost_fp32"] else r1
    assert best["cost_fp32"] == rw["cost_fp32"] and best["cost_fp64"] == rw["cost_fp64"]
    np.testing.assert_array_equal(best["hubs"], rw["hubs"])


def test_exchange_calls_check_their_arguments():
    inst = synth.urand200(seed=58, n=40, p=4)
    with Instance.from_instance(inst) as gi:
        with pytest.raises(UsaphmpError):
            gi.ga_islands()                              # before ga_begin
        with pytest.raises(UsaphmpError):
            gi.set_params(island_offset=-1)
        with pytest.raises(UsaphmpError):
            gi.set_params(islands=4, island_size=64, island_offset=(1 << 31) // 64)
        gi.set_params(islands=2, island_size=8, n1=0)
        gi.ga_begin(1)
        masks, fit = gi.ga_islands()
        assert masks.shape == (2, gi.nw) and fit.shape == (2,)
        bad = masks[0].copy()
        bad[0] ^= 1 << 31 if inst.n > 32 else 0
        bad[-1] |= np.uint32(1 << 31) if inst.n % 32 else 0
        with pytest.raises(UsaphmpError):
            gi.ga_merge(bad, 1.0)                        # not p hubs among the first n nodes
        gi.ga_merge(masks[1], fit[1])
        m2, f2 = gi.ga_islands()
        np.testing.assert_array_equal(m2, np.stack([masks[1], masks[1]]))
        assert (f2 == fit[1]).all()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SHARD_CASES = {
    "small_plain": dict(n=180, p=7, inst_seed=57, seed=31, R=3, P=16, N1=4, G=12, path=PATH_PLAIN_FP32),
    "small_split": dict(n=180, p=7, inst_seed=57, seed=31, R=3, P=16, N1=4, G=12, path=PATH_SPLIT_BF16),
    # the bench shape (64 islands x 64, clustered n=1000, p=20) split over two ranks
    "bench_split": dict(n=1000, p=20, inst_seed=1003, seed=4321, R=32, P=64, N1=2, G=5, path=PATH_SPLIT_BF16),
}


@pytest.mark.parametrize("case", list(SHARD_CASES), ids=list(SHARD_CASES))
def test_sharded_solve_on_two_processes_follows_one_handle_and_the_oracle(case, tmp_path):
    """dist.sharded_solve itself, on two spawned processes (gloo exchange,
    both on cuda:0): every generation's children and fitness, the ancestors
    after each selection and after each cross-rank merge, and the final result
    equal one handle holding every island; the shards' children are the
    oracle's make_children(island_offset) of the oracle's own shard states,
    which select on the GPU's fitness and merge by merge_shards."""
    import multiprocessing as mp

    import shard_worker
    from oracle import ga
    from gpu_util import unpack_masks

    c = SHARD_CASES[case]
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=shard_worker.run, args=(k, world, port, str(tmp_path), c)) for k in range(world)]
    for pr in procs:
        pr.start()
    try:
        for pr in procs:
            pr.join(timeout=600)
        assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
    finally:
        for pr in procs:
            if pr.is_alive():
                pr.kill()
    tr = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    inst = synth.clustered(seed=c["inst_seed"], n=c["n"], p=c["p"])
    n, p, R, P, N1, G, seed = inst.n, inst.p, c["R"], c["P"], c["N1"], c["G"], c["seed"]

    # one handle holding every island, generation by generation
    with Instance.from_instance(inst) as whole:
        whole.set_params(islands=world * R, island_size=P, n1=N1, path=c["path"])
        whole.ga_begin(seed)
        m0, f0 = whole.ga_islands()
        merge_k = 0
        for g in range(G):
            whole.ga_run(1)
            wm, wf = whole.ga_population()
            np.testing.assert_array_equal(np.concatenate([t["children"][g] for t in tr]), wm)
            np.testing.assert_array_equal(np.concatenate([t["fit"][g] for t in tr]), wf)
            am, af = whole.ga_islands()
            if (g + 1) % N1 == 0:
                for t in tr:
                    assert t["merge_g"][merge_k] == g
                    np.testing.assert_array_equal(t["merge_anc"][merge_k], am[:R])
                    np.testing.assert_array_equal(t["merge_anc_fit"][merge_k], af[:R])
                merge_k += 1
            else:
                np.testing.assert_array_equal(np.concatenate([t["anc"][g] for t in tr]), am)
                np.testing.assert_array_equal(np.concatenate([t["anc_fit"][g] for t in tr]), af)
        rw = whole.ga_result()
    assert merge_k == len(tr[0]["merge_g"]) == G // N1
    for t in tr:
        np.testing.assert_array_equal(t["hubs"], rw["hubs"])
        np.testing.assert_array_equal(t["S"], rw["S"])
        assert t["cost"][0] == rw["cost_fp64"] and np.float32(t["cost"][1]) == np.float32(rw["cost_fp32"])

    # the oracle's shards, fed the GPU's fitness
    anc0 = unpack_masks(m0, n)
    st = [ga.State(anc0[k * R:(k + 1) * R], f0[k * R:(k + 1) * R].astype(np.float64), anc0[0], float(f0[0]))
          for k in range(world)]
    merge_k = 0
    for g in range(G):
        for k in range(world):
            children = ga.make_children(st[k].ancestors, seed, g, p, P, island_offset=k * R)
            np.testing.assert_array_equal(unpack_masks(tr[k]["children"][g], n), children)
            ga.select(st[k], children, tr[k]["fit"][g].astype(np.float64), g, P, 0)
            np.testing.assert_array_equal(unpack_masks(tr[k]["anc"][g], n), st[k].ancestors)
            np.testing.assert_array_equal(tr[k]["anc_fit"][g], st[k].anc_fit.astype(np.float32))
        if (g + 1) % N1 == 0:
            wmask, wfit = ga.merge_shards(st, [R] * world)
            for k in range(world):
                np.testing.assert_array_equal(unpack_masks(tr[k]["merge_mask"][merge_k][None], n)[0], wmask)
                assert tr[k]["merge_fit"][merge_k] == np.float32(wfit)
            merge_k += 1

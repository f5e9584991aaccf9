"""Allocation local search (fp64 single reallocations) through the C ABI,
bit-exact against the oracle's search."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, stream, torch
from oracle import brute, cost
from oracle.local_search import local_search
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import (PATH_PLAIN_FP32, PATH_SPLIT_BF16, ROUTE_DIRECT, ROUTE_HUB_PATHS,
                                            Instance, UsaphmpError)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def heavy_tailed(seed, n, p, spread=0.0):
    """Flows with a heavy tail: the nearest hub is then often not the best."""
    inst = synth.latency_like(seed=seed, n=n, p=p, spread=spread)
    rng = np.random.default_rng(seed)
    W = (inst.W * rng.lognormal(0.0, 1.5, size=inst.W.shape)).astype(np.float32)
    np.fill_diagonal(W, 0.0)
    return synth.Instance(f"heavy{n}", n, p, W, inst.C)


def run_gpu(gi, hubs, S, max_sweeps):
    B = len(hubs)
    hs = np.sort(hubs, axis=1).astype(np.int32)
    slot = np.full((B, gi.ns), 255, np.uint8)
    for b in range(B):
        slot[b, :gi.n] = cost.slots_of(hs[b], S[b])
    d_hs, d_slot = dev(hs), dev(slot)
    mv = torch.zeros(B, dtype=torch.int32, device="cuda")
    sw = torch.zeros(B, dtype=torch.int32, device="cuda")
    gi.local_search_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), max_sweeps, mv.data_ptr(), sw.data_ptr(), stream())
    out = host(d_slot)[:, :gi.n].astype(np.int64)
    return np.take_along_axis(hs.astype(np.int64), out, axis=1), host(mv), host(sw), d_hs, d_slot


@pytest.mark.parametrize("seed,n,p,routing", [(5, 40, 3, "direct"), (9, 61, 5, "direct"), (25, 80, 12, "direct"),
                                              (41, 50, 4, "hubs"), (43, 70, 9, "hubs"), (45, 33, 1, "direct"),
                                              # several candidate warps; hub table in global memory at p = 150
                                              (61, 100, 70, "direct"), (65, 90, 40, "hubs"), (63, 170, 150, "direct")])
def test_search_matches_oracle(seed, n, p, routing):
    inst = heavy_tailed(seed, n, p, spread=0.8 if routing == "hubs" else 0.0)
    rng = np.random.default_rng(seed)
    B = 6
    hubs = np.stack([np.sort(rng.choice(n, p, replace=False)) for _ in range(B)])
    starts = []
    for b in range(B):
        s = cost.nearest_allocation(inst.C, hubs[b]) if b % 2 == 0 else hubs[b][rng.integers(0, p, size=n)]
        s = s.copy()
        s[hubs[b]] = hubs[b]
        starts.append(s)
    starts = np.stack(starts)
    with Instance.from_instance(inst) as gi:
        gi.set_params(routing=ROUTE_HUB_PATHS if routing == "hubs" else ROUTE_DIRECT)
        got, moves, sweeps, _, _ = run_gpu(gi, hubs, starts, 10)
    total = 0
    for b in range(B):
        ref, rs, rm = local_search(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, hubs[b], starts[b], 10, routing)
        np.testing.assert_array_equal(got[b], ref, err_msg=f"chromosome {b}")
        assert (moves[b], sweeps[b]) == (rm, rs)
        total += rm
    assert p == 1 or total > 0


def test_improves_and_converges_at_bench_size():
    inst = synth.clustered()
    B = 6
    hubs, _ = synth.random_population(7, inst.n, inst.p, B)
    hubs = np.sort(hubs, axis=1)
    S = np.stack([cost.nearest_allocation(inst.C, h) for h in hubs])
    with Instance.from_instance(inst) as gi:
        got, moves, sweeps, d_hs, d_slot = run_gpu(gi, hubs, S, 50)
        assert (sweeps < 50).all() and (moves > 0).any()
        c = torch.empty(B, dtype=torch.float64, device="cuda")
        gi.rescore_fp64_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), c.data_ptr(), stream())
        after = host(c)
        again, moves2, sweeps2, _, _ = run_gpu(gi, hubs, got, 50)
    np.testing.assert_array_equal(again, got)          # a fixed point
    assert (moves2 == 0).all() and (sweeps2 == 1).all()
    for b in range(B):
        cost.check_allocation(inst.n, hubs[b], got[b])
        before = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, S[b])
        ref_after = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, got[b])
        assert after[b] == pytest.approx(ref_after, rel=1e-12)
        assert ref_after <= before


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_solve_returns_the_searched_allocation(path):
    inst = heavy_tailed(9, 10, 3)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=1, island_size=64, n1=10, path=path)
        plain = gi.solve(100, 2024)
        gi.set_params(local_search=10)
        r = gi.solve(100, 2024)
    np.testing.assert_array_equal(r["hubs"], plain["hubs"])        # the search runs after the GA
    near = cost.nearest_allocation(inst.C, r["hubs"])
    np.testing.assert_array_equal(plain["S"], near)
    ref, _, _ = local_search(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, r["hubs"], near, 10)
    np.testing.assert_array_equal(r["S"], ref)
    ref_cost = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, ref)
    assert r["cost_fp64"] == pytest.approx(ref_cost, rel=1e-12)
    assert r["cost_fp64"] <= plain["cost_fp64"]
    assert abs(r["cost_fp32"] - r["cost_fp64"]) / r["cost_fp64"] <= 1e-4
    bf = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p)
    assert r["cost_fp64"] >= bf["opt"][0] * (1 - 1e-12)


def test_bad_arguments():
    inst = heavy_tailed(3, 20, 3)
    with Instance.from_instance(inst) as gi:
        with pytest.raises(UsaphmpError):
            gi.set_params(local_search=-1)
        with pytest.raises(UsaphmpError):
            gi.local_search_dev(1, 0, 0, 1)


def test_search_matches_oracle_without_fp32_screen():
    """p = 220: the fp32 hub table no longer fits in shared memory, so every
    spoke is decided by the fp64 evaluation alone."""
    seed, n, p = 67, 236, 220
    inst = heavy_tailed(seed, n, p)
    rng = np.random.default_rng(seed)
    hubs = np.stack([np.sort(rng.choice(n, p, replace=False)) for _ in range(2)])
    starts = []
    for b in range(2):
        s = cost.nearest_allocation(inst.C, hubs[b]) if b == 0 else hubs[b][rng.integers(0, p, size=n)]
        s = s.copy()
        s[hubs[b]] = hubs[b]
        starts.append(s)
    starts = np.stack(starts)
    with Instance.from_instance(inst) as gi:
        got, moves, sweeps, _, _ = run_gpu(gi, hubs, starts, 3)
    for b in range(2):
        ref, rs, rm = local_search(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, hubs[b], starts[b], 3)
        np.testing.assert_array_equal(got[b], ref, err_msg=f"chromosome {b}")
        assert (moves[b], sweeps[b]) == (rm, rs)


def _oracle_pool(inst):
    """Spawned oracle workers (no CUDA state) holding the instance."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor

    import oracle_workers
    return ProcessPoolExecutor(min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn"),
                               initializer=oracle_workers.init,
                               initargs=(inst.W, inst.C, inst.chi, inst.alpha, inst.delta))


def test_search_matches_oracle_at_n400():
    """Whole searches at n = 400 against the oracle's (which evaluates every
    candidate move as a difference of two pair-form costs): allocations,
    moves and sweeps, from a nearest and from a random allocation."""
    import oracle_workers
    seed, n, p = 71, 400, 6
    inst = heavy_tailed(seed, n, p)
    rng = np.random.default_rng(seed)
    hubs = np.stack([np.sort(rng.choice(n, p, replace=False)) for _ in range(2)])
    starts = []
    for b in range(2):
        s = cost.nearest_allocation(inst.C, hubs[b]) if b == 0 else hubs[b][rng.integers(0, p, size=n)]
        s = s.copy()
        s[hubs[b]] = hubs[b]
        starts.append(s)
    starts = np.stack(starts)
    with _oracle_pool(inst) as pool:
        refs = pool.map(oracle_workers.run_local_search, [(hubs[b], starts[b], 20, "direct") for b in range(2)])
        with Instance.from_instance(inst) as gi:
            got, moves, sweeps, _, _ = run_gpu(gi, hubs, starts, 20)
        refs = list(refs)
    for b, (ref, rs, rm) in enumerate(refs):
        np.testing.assert_array_equal(got[b], ref, err_msg=f"chromosome {b}")
        assert (moves[b], sweeps[b]) == (rm, rs)
    assert moves.sum() > 0


def test_bench_size_result_is_a_local_optimum_sampled():
    """At the bench size (clustered n = 1000, p = 20) the search's result, for
    32 sampled spokes of each of 4 chromosomes, admits no improving single
    reallocation by the oracle's pair-form costs, and the fp64 cost the GPU
    returns for it equals the oracle's."""
    import oracle_workers
    inst = synth.clustered()
    B, per = 4, 32
    hubs, _ = synth.random_population(11, inst.n, inst.p, B)
    hubs = np.sort(hubs, axis=1)
    S = np.stack([cost.nearest_allocation(inst.C, h) for h in hubs])
    with Instance.from_instance(inst) as gi:
        got, moves, sweeps, d_hs, d_slot = run_gpu(gi, hubs, S, 50)
        c = torch.empty(B, dtype=torch.float64, device="cuda")
        gi.rescore_fp64_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), c.data_ptr(), stream())
        gpu_cost = host(c)
    assert (sweeps < 50).all() and (moves > 0).any()
    rng = np.random.default_rng(12)
    jobs = []
    for b in range(B):
        spokes = np.setdiff1d(np.arange(inst.n), hubs[b])
        for i in rng.choice(spokes, per, replace=False):
            jobs.append((got[b], int(i), hubs[b]))
    with _oracle_pool(inst) as pool:
        out = list(pool.map(oracle_workers.single_move_changes, jobs, chunksize=4))
    for k, (changes, base) in enumerate(out):
        b = k // per
        assert gpu_cost[b] == pytest.approx(base, rel=1e-12)
        # a change the two fp64 sums cannot tell from zero is no improvement
        worst = min(d for _, d in changes)
        assert worst >= -1e-13 * base, (b, jobs[k][1], worst)

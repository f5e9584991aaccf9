"""Hub-path routing of the transfer leg (eq. 4) on non-metric costs, through
the C ABI, against the FP64 oracle with routing="hubs"."""
import zlib

import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, stream, torch, unpack_masks
from oracle import brute, cost, ga
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import (PATH_PLAIN_FP32, PATH_SPLIT_BF16, ROUTE_DIRECT, ROUTE_HUB_PATHS,
                                            Instance, UsaphmpError)

pytestmark = pytest.mark.gpu

TOL = {PATH_PLAIN_FP32: 1e-5, PATH_SPLIT_BF16: 1e-4}
PATHS = [PATH_PLAIN_FP32, PATH_SPLIT_BF16]

CASES = {
    "n200_p10": lambda: synth.latency_like(seed=61, n=200, p=10),
    "n333_p7_ragged": lambda: synth.latency_like(seed=62, n=333, p=7),
    "n150_p20": lambda: synth.latency_like(seed=63, n=150, p=20, spread=1.0),
    "n300_p63": lambda: synth.latency_like(seed=64, n=300, p=63),
    "n260_p100": lambda: synth.latency_like(seed=65, n=260, p=100),
    "n300_p150_global_table": lambda: synth.latency_like(seed=73, n=300, p=150),
    "n12_p1": lambda: synth.latency_like(seed=66, n=12, p=1),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def oracle_costs(inst, S, routing):
    return np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s, routing) for s in S])


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_hub_paths_match_oracle(case, path):
    inst = CASES[case]()
    B = 29
    hubs, S = synth.random_population(zlib.crc32(case.encode()) % 1000, inst.n, inst.p, B)
    ref = oracle_costs(inst, S, "hubs")
    direct = oracle_costs(inst, S, "direct")
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path, routing=ROUTE_HUB_PATHS)
        got = gi.eval(hubs, S)
        gi.set_params(routing=ROUTE_DIRECT)
        got_direct = gi.eval(hubs, S)
    assert (np.abs(got - ref) / ref).max() <= TOL[path]
    assert (np.abs(got_direct - direct) / direct).max() <= TOL[path]
    if inst.p > 2:
        assert (ref < direct * (1 - 1e-6)).any()        # the instance does reward detours


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
def test_hub_paths_change_nothing_on_euclidean_costs(path):
    inst = synth.urand200(seed=67, n=250, p=12)
    hubs, S = synth.random_population(68, inst.n, inst.p, 16)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        a = gi.eval(hubs, S)
        gi.set_params(routing=ROUTE_HUB_PATHS)
        b = gi.eval(hubs, S)
    np.testing.assert_allclose(b, a, rtol=1e-6)


def test_rescore_fp64_with_hub_paths():
    inst = synth.latency_like(seed=69, n=240, p=9, spread=1.0)
    B = 5
    hubs, S = synth.random_population(70, inst.n, inst.p, B)
    ref = oracle_costs(inst, S, "hubs")
    with Instance.from_instance(inst) as gi:
        gi.set_params(routing=ROUTE_HUB_PATHS)
        hs = np.sort(hubs, axis=1).astype(np.int32)
        slot = np.full((B, gi.ns), 255, np.uint8)
        for b in range(B):
            slot[b, :inst.n] = cost.slots_of(hs[b], S[b])
        c = torch.empty(B, dtype=torch.float64, device="cuda")
        d_hs, d_slot = dev(hs), dev(slot)
        gi.rescore_fp64_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), c.data_ptr(), stream())
        got = host(c)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
def test_solve_reaches_the_routed_brute_force_nearest_optimum(path):
    inst = synth.latency_like(seed=71, n=10, p=3, spread=1.0)
    bf = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p, routing="hubs")
    direct = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p)
    assert bf["nearest"][0] < direct["nearest"][0]
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=1, island_size=64, n1=10, path=path, routing=ROUTE_HUB_PATHS)
        r = gi.solve(100, 2024)
    assert r["cost_fp64"] == pytest.approx(bf["nearest"][0], rel=1e-12)
    cost.check_allocation(inst.n, r["hubs"], r["S"])
    assert r["cost_fp64"] == pytest.approx(
        cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, r["S"], "hubs"), rel=1e-12)
    assert abs(r["cost_fp32"] - r["cost_fp64"]) / r["cost_fp64"] <= TOL[path]


def test_unknown_routing_is_refused():
    inst = synth.latency_like(seed=72, n=20, p=3)
    with Instance.from_instance(inst) as gi:
        with pytest.raises(UsaphmpError) as e:
            gi.set_params(routing=2)
        assert e.value.name == "EINVAL"
        assert gi.params["routing"] == ROUTE_DIRECT


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
def test_ga_run_with_hub_paths_follows_the_oracle(path):
    """Graph-replayed generations with hub-path routing (the block allocation
    kernel relaxes every chromosome's hub table): children equal the oracle's,
    fitness within the path's tolerance of the oracle's routed objective, and
    the ancestors after selection equal the oracle's, generation by generation."""
    n, p, R, P, N1, seed, G = 150, 12, 2, 16, 2, 4141, 3
    inst = synth.latency_like(seed=74, n=n, p=p, spread=1.0)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path, routing=ROUTE_HUB_PATHS, use_graph=1)
        gi.ga_begin(seed)
        am, af = gi.ga_islands()
        st = ga.State(unpack_masks(am, n), af.astype(np.float64), unpack_masks(am, n)[0], float(af[0]))
        for g in range(G):
            gi.ga_run(1)
            masks, fit = gi.ga_population()
            children = ga.make_children(st.ancestors, seed, g, p, P)
            np.testing.assert_array_equal(unpack_masks(masks, n), children)
            _, hh, _ = ga.allocate_all(inst.C, children)
            ref = oracle_costs(inst, hh, "hubs")
            assert (np.abs(fit - ref) / ref).max() <= TOL[path]
            ga.select(st, children, fit.astype(np.float64), g, P, N1)
            am, af = gi.ga_islands()
            np.testing.assert_array_equal(unpack_masks(am, n), st.ancestors)

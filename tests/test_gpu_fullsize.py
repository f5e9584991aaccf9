"""Parity at the full workload sizes, in the launch configuration bench.py times.

The population shapes of the benchmark configurations are evaluated whole on
the GPU; the oracle checks every chromosome where it finishes in seconds and
a seeded sample otherwise.
"""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, pack_masks, stream, torch, unpack_masks
from oracle import cost, ga
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance

pytestmark = pytest.mark.gpu
TOL = {PATH_PLAIN_FP32: 1e-5, PATH_SPLIT_BF16: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _rel(inst, S, got, idx):
    ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, S[b]) for b in idx])
    return np.abs(got[idx] - ref) / ref


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
@pytest.mark.parametrize("p", [5, 10, 20])
def test_urand200_population_1024_all_chromosomes(p, path):
    inst = synth.urand200(p=p)
    hubs, S = synth.random_population(300 + p, inst.n, inst.p, 1024)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        got = gi.eval(hubs, S)
    assert _rel(inst, S, got, np.arange(1024)).max() <= TOL[path]


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_clustered1000_population_4096_sampled(path):
    inst = synth.clustered()
    hubs, S = synth.random_population(400, inst.n, inst.p, 4096)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        got = gi.eval(hubs, S)
    idx = np.random.default_rng(401).choice(4096, 48, replace=False)
    idx = np.concatenate([idx, [0, 4095]])
    assert _rel(inst, S, got, idx).max() <= TOL[path]


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
@pytest.mark.parametrize("p", [20, 50])
def test_uniform6000_population_2048_sampled(p, path):
    inst = synth.large_uniform(p=p)
    hubs, S = synth.random_population(500 + p, inst.n, inst.p, 2048)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        got = gi.eval(hubs, S)
    idx = np.array([0, 777, 2047])
    assert _rel(inst, S, got, idx).max() <= TOL[path]


def test_clustered1000_ga_generation_bit_exact_sampled():
    """One generation of the bench workload (64 islands x 64) on the GPU against
    the oracle: every child mask, and the allocation of a sample."""
    inst = synth.clustered()
    R, P, seed, g = 64, 64, 1234, 3
    B = R * P
    anc = synth.random_masks(402, inst.n, inst.p, R)
    ref = ga.make_children(anc, seed, g, inst.p, P)
    with Instance.from_instance(inst) as gi:
        d_anc = dev(pack_masks(anc).view(np.int32))
        m = torch.zeros((B, gi.nw), dtype=torch.int32, device="cuda")
        h = torch.zeros((B, inst.p), dtype=torch.int32, device="cuda")
        sl = torch.zeros((B, gi.ns), dtype=torch.uint8, device="cuda")
        gi.children_dev(R, P, d_anc.data_ptr(), seed, g, m.data_ptr(), h.data_ptr(), stream())
        gi.allocate_dev(B, h.data_ptr(), sl.data_ptr(), stream())
        got = unpack_masks(host(m).view(np.uint32), inst.n)
        slots = host(sl)
    np.testing.assert_array_equal(got, ref)
    for b in np.random.default_rng(403).choice(B, 24, replace=False):
        hb = np.flatnonzero(ref[b])
        np.testing.assert_array_equal(slots[b, :inst.n], cost.slots_of(hb, cost.nearest_allocation(inst.C, hb)))


def test_clustered1000_graph_generations_follow_the_oracle():
    """The benchmarked path itself -- 64 islands x 64 on clustered n=1000, p=20,
    split-bf16, generations replayed from the CUDA graph with the fused
    reduction + selection -- one generation at a time: every child mask, the
    ancestors and their fitness after every selection (a merge every second
    generation) and the final best-ever against the oracle's GA fed the GPU's
    fitness; sampled fitness against the fp64 objective."""
    inst = synth.clustered()
    n, p = inst.n, inst.p
    R, P, N1, seed, G = 64, 64, 2, 4321, 3
    B = R * P
    rng = np.random.default_rng(404)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=PATH_SPLIT_BF16, use_graph=1)
        gi.ga_begin(seed)
        am, af = gi.ga_islands()
        m0 = np.isin(np.arange(n), cost.middle_nodes(inst.C, p))
        np.testing.assert_array_equal(unpack_masks(am, n), np.tile(m0, (R, 1)))
        assert (af == af[0]).all()
        st = ga.State(np.tile(m0, (R, 1)), af.astype(np.float64), m0, float(af[0]))
        for g in range(G):
            gi.ga_run(1)
            masks, fit = gi.ga_population()
            children = ga.make_children(st.ancestors, seed, g, p, P)
            np.testing.assert_array_equal(unpack_masks(masks, n), children)
            for b in rng.choice(B, 6, replace=False):
                h = cost.nearest_allocation(inst.C, np.flatnonzero(children[b]))
                ref = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, h)
                assert abs(fit[b] - ref) / ref <= TOL[PATH_SPLIT_BF16]
            ga.select(st, children, fit.astype(np.float64), g, P, N1)
            am, af = gi.ga_islands()
            np.testing.assert_array_equal(unpack_masks(am, n), st.ancestors)
            np.testing.assert_array_equal(af, st.anc_fit.astype(np.float32))
        res = gi.ga_result()
    np.testing.assert_array_equal(res["hubs"], np.flatnonzero(st.best))
    assert np.float32(res["cost_fp32"]) == np.float32(st.best_fit)

"""GPU GA step vs the oracle: bit-exact masks, hubs, slots and selection."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, pack_masks, stream, torch, unpack_masks
from oracle import brute, cost, ga
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("n,p", [(10, 3), (200, 20), (333, 7), (1000, 20)])
def test_initial_solution_is_middle_nodes(n, p):
    inst = synth.urand200(seed=n, n=n, p=p) if n < 1000 else synth.clustered()
    with Instance.from_instance(inst) as gi:
        m = torch.zeros(gi.nw, dtype=torch.int32, device="cuda")
        h = torch.zeros(p, dtype=torch.int32, device="cuda")
        gi.initial_dev(m.data_ptr(), h.data_ptr(), stream())
        hubs = host(h)
        mask = unpack_masks(host(m).view(np.uint32)[None], n)[0]
    ref = cost.middle_nodes(inst.C, p)
    np.testing.assert_array_equal(hubs, ref)
    np.testing.assert_array_equal(np.flatnonzero(mask), ref)


def _lattice(side, seed=0):
    """Nodes on a side x side unit grid: symmetric nodes have rows of C that
    are permutations of each other, so their middle-node scores tie exactly."""
    xy = np.stack(np.meshgrid(np.arange(side), np.arange(side), indexing="ij"), -1).reshape(-1, 2).astype(np.float64)
    d = xy[:, None, :] - xy[None, :, :]
    C = np.sqrt((d ** 2).sum(-1)).astype(np.float32)
    W = np.random.default_rng(seed).uniform(0, 1, C.shape).astype(np.float32)
    np.fill_diagonal(W, 0.0)
    return W, C


@pytest.mark.parametrize("side,p", [(9, 1), (9, 4), (9, 9), (12, 1), (12, 6), (12, 10)])
def test_initial_solution_ties_on_a_lattice(side, p):
    W, C = _lattice(side)
    n = side * side
    inst = synth.Instance(f"lattice{side}", n, p, W, C)
    with Instance.from_instance(inst) as gi:
        m = torch.zeros(gi.nw, dtype=torch.int32, device="cuda")
        h = torch.zeros(p, dtype=torch.int32, device="cuda")
        gi.initial_dev(m.data_ptr(), h.data_ptr(), stream())
        hubs = host(h)
        mask = unpack_masks(host(m).view(np.uint32)[None], n)[0]
    ref = cost.middle_nodes(C, p)
    np.testing.assert_array_equal(hubs, ref)
    np.testing.assert_array_equal(np.flatnonzero(mask), ref)


@pytest.mark.parametrize("n,p,B", [(10, 3, 16), (200, 10, 64), (333, 7, 40), (1000, 20, 24), (64, 64, 3)])
def test_allocation_bit_exact(n, p, B):
    inst = synth.urand200(seed=n + 1, n=n, p=p) if n != 1000 else synth.clustered()
    masks = synth.random_masks(n + p, n, p, B)
    hubs = np.stack([np.flatnonzero(m) for m in masks]).astype(np.int32)
    with Instance.from_instance(inst) as gi:
        slot = torch.zeros((B, gi.ns), dtype=torch.uint8, device="cuda")
        d_hubs = dev(hubs)
        gi.allocate_dev(B, d_hubs.data_ptr(), slot.data_ptr(), stream())
        got = host(slot)
    for b in range(B):
        ref = cost.slots_of(hubs[b], cost.nearest_allocation(inst.C, hubs[b]))
        np.testing.assert_array_equal(got[b, :n], ref)
        assert (got[b, n:] == 255).all()


def test_allocation_ties_go_to_lowest_node():
    # clustered duplicate points: many exact distance ties
    rng = np.random.default_rng(5)
    base = rng.uniform(0, 10, (6, 2))
    xy = base[rng.integers(0, 6, 90)]
    d = xy[:, None, :] - xy[None, :, :]
    C = np.sqrt((d ** 2).sum(-1)).astype(np.float32)
    W = rng.uniform(0, 1, (90, 90)).astype(np.float32)
    inst = synth.Instance("ties", 90, 8, W, C)
    masks = synth.random_masks(6, 90, 8, 32)
    hubs = np.stack([np.flatnonzero(m) for m in masks]).astype(np.int32)
    with Instance.from_instance(inst) as gi:
        slot = torch.zeros((32, gi.ns), dtype=torch.uint8, device="cuda")
        d_hubs = dev(hubs)
        gi.allocate_dev(32, d_hubs.data_ptr(), slot.data_ptr(), stream())
        got = host(slot)
    for b in range(32):
        ref = cost.slots_of(hubs[b], cost.nearest_allocation(C, hubs[b]))
        np.testing.assert_array_equal(got[b, :90], ref)


@pytest.mark.parametrize("n,p,R,P,seed,g", [
    (10, 3, 1, 64, 2024, 0), (10, 3, 2, 8, 7, 5), (50, 5, 3, 8, 99, 4), (200, 20, 2, 64, 1, 123),
    (333, 7, 4, 6, 31337, 9), (1000, 20, 2, 16, 2**40 + 5, 77), (64, 63, 1, 4, 3, 0), (97, 1, 2, 4, 8, 2),
])
def test_children_bit_exact(n, p, R, P, seed, g):
    inst = synth.urand200(seed=n, n=n, p=p)
    anc = synth.random_masks(seed % 1000 + n, n, p, R)
    ref = ga.make_children(anc, seed, g, p, P)
    with Instance.from_instance(inst) as gi:
        B = R * P
        m = torch.zeros((B, gi.nw), dtype=torch.int32, device="cuda")
        h = torch.zeros((B, p), dtype=torch.int32, device="cuda")
        d_anc = dev(pack_masks(anc).view(np.int32))
        gi.children_dev(R, P, d_anc.data_ptr(), seed, g, m.data_ptr(),
                        h.data_ptr(), stream())
        got = unpack_masks(host(m).view(np.uint32), n)
        hubs = host(h)
    np.testing.assert_array_equal(got, ref)
    for b in range(B):
        np.testing.assert_array_equal(hubs[b], np.flatnonzero(ref[b]))


def _select_case(R, P, nw, rng, ties):
    fit = rng.uniform(10, 20, R * P).astype(np.float32)
    if ties == "nan":
        fit[rng.random(R * P) < 0.5] = np.nan
        fit[:P] = np.nan            # an island with no number at all
    elif ties:
        fit = np.round(fit).astype(np.float32)
    return fit


@pytest.mark.parametrize("R,P,g,N1,ties,elitist", [
    (4, 8, 0, 10, False, 0), (4, 8, 9, 10, True, 0), (7, 6, 19, 5, True, 0), (3, 64, 2, 3, False, 1),
    (5, 4, 4, 5, True, 1), (4, 8, 9, 10, "nan", 0),
])
def test_selection_bit_exact(R, P, g, N1, ties, elitist):
    n, p = 70, 5
    inst = synth.urand200(seed=3, n=n, p=p)
    rng = np.random.default_rng(R * 100 + g)
    children = synth.random_masks(g + 1, n, p, R * P)
    anc = synth.random_masks(g + 2, n, p, R)
    fit = _select_case(R, P, None, rng, ties)
    anc_fit = rng.uniform(9, 21, R).astype(np.float32)
    best = synth.random_masks(g + 3, n, p, 1)[0]
    best_fit = np.float32(12.5)
    st = ga.State(anc, anc_fit.astype(np.float64), best, float(best_fit))
    ga.select(st, children, fit.astype(np.float64), g, P, N1, elitist=bool(elitist))
    with Instance.from_instance(inst) as gi:
        gi.set_params(n1=N1, elitist=elitist)
        d_anc = dev(pack_masks(anc).view(np.int32))
        d_af = dev(anc_fit)
        d_best = dev(pack_masks(best).view(np.int32)[0])
        d_bf = dev(np.array([best_fit], np.float32))
        d_children, d_fit = dev(pack_masks(children).view(np.int32)), dev(fit)
        gi.select_dev(R, P, g, d_children.data_ptr(), d_fit.data_ptr(),
                      d_anc.data_ptr(), d_af.data_ptr(), d_best.data_ptr(), d_bf.data_ptr(), stream())
        got_anc = unpack_masks(host(d_anc).view(np.uint32), n)
        got_af = host(d_af)
        got_best = unpack_masks(host(d_best).view(np.uint32)[None], n)[0]
        got_bf = host(d_bf)[0]
    np.testing.assert_array_equal(got_anc, st.ancestors)
    np.testing.assert_array_equal(got_af, st.anc_fit.astype(np.float32))
    np.testing.assert_array_equal(got_best, st.best)
    assert got_bf == np.float32(st.best_fit)


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_ga_generations_replay_bit_exact(path):
    """G generations on the GPU, each step checked against the oracle fed the GPU's fitness."""
    n, p, R, P, N1, seed, G = 120, 6, 3, 8, 3, 4242, 7
    inst = synth.urand200(seed=15, n=n, p=p)
    B = R * P
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path)
        anc = np.tile(np.isin(np.arange(n), cost.middle_nodes(inst.C, p)), (R, 1))
        st = ga.State(anc, np.full(R, 1e30), anc[0], 1e30)
        d_anc = dev(pack_masks(anc).view(np.int32))
        d_af = dev(np.full(R, 1e30, np.float32))
        d_best = dev(pack_masks(anc[0]).view(np.int32)[0])
        d_bf = dev(np.array([1e30], np.float32))
        m = torch.zeros((B, gi.nw), dtype=torch.int32, device="cuda")
        h = torch.zeros((B, p), dtype=torch.int32, device="cuda")
        sl = torch.zeros((B, gi.ns), dtype=torch.uint8, device="cuda")
        f = torch.zeros(B, dtype=torch.float32, device="cuda")
        for g in range(G):
            gi.children_dev(R, P, d_anc.data_ptr(), seed, g, m.data_ptr(), h.data_ptr(), stream())
            gi.allocate_dev(B, h.data_ptr(), sl.data_ptr(), stream())
            gi.eval_slots_dev(B, h.data_ptr(), sl.data_ptr(), f.data_ptr(), stream())
            fit = host(f)
            children = ga.make_children(st.ancestors, seed, g, p, P)
            np.testing.assert_array_equal(unpack_masks(host(m).view(np.uint32), n), children)
            _, hh, slot = ga.allocate_all(inst.C, children)
            np.testing.assert_array_equal(host(sl)[:, :n], slot)
            ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, x) for x in hh])
            assert (np.abs(fit - ref) / ref).max() <= (1e-5 if path == PATH_PLAIN_FP32 else 1e-4)
            ga.select(st, children, fit.astype(np.float64), g, P, N1)
            gi.select_dev(R, P, g, m.data_ptr(), f.data_ptr(), d_anc.data_ptr(), d_af.data_ptr(),
                          d_best.data_ptr(), d_bf.data_ptr(), stream())
            np.testing.assert_array_equal(unpack_masks(host(d_anc).view(np.uint32), n), st.ancestors)
            np.testing.assert_array_equal(unpack_masks(host(d_best).view(np.uint32)[None], n)[0], st.best)


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_fused_generation_equals_step_chain(path, use_graph):
    """The GA loop (fused reduction + selection, optionally graph-replayed)
    gives the same state as the step-level kernels (separate reduction and
    selection)."""
    n, p, R, P, N1, seed, G = 230, 9, 4, 16, 3, 77, 8
    inst = synth.clustered(seed=16, n=n, p=p)
    B = R * P
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path, use_graph=use_graph)
        gi.ga_begin(seed, stream())
        gi.ga_run(G, stream())
        fused = gi.ga_result(stream())
        # the same generations through the step-level entry points
        hubs0 = cost.middle_nodes(inst.C, p).astype(np.int32)
        m0 = np.isin(np.arange(n), hubs0)
        d_h0 = dev(hubs0[None])
        s0 = torch.zeros((1, gi.ns), dtype=torch.uint8, device="cuda")
        f0 = torch.zeros(1, dtype=torch.float32, device="cuda")
        gi.allocate_dev(1, d_h0.data_ptr(), s0.data_ptr(), stream())
        gi.eval_slots_dev(1, d_h0.data_ptr(), s0.data_ptr(), f0.data_ptr(), stream())
        fit0 = float(host(f0)[0])
        d_anc = dev(pack_masks(np.tile(m0, (R, 1))).view(np.int32))
        d_af = dev(np.full(R, fit0, np.float32))
        d_best = dev(pack_masks(m0).view(np.int32)[0])
        d_bf = dev(np.array([fit0], np.float32))
        m = torch.zeros((B, gi.nw), dtype=torch.int32, device="cuda")
        h = torch.zeros((B, p), dtype=torch.int32, device="cuda")
        sl = torch.zeros((B, gi.ns), dtype=torch.uint8, device="cuda")
        f = torch.zeros(B, dtype=torch.float32, device="cuda")
        for g in range(G):
            gi.children_dev(R, P, d_anc.data_ptr(), seed, g, m.data_ptr(), h.data_ptr(), stream())
            gi.allocate_dev(B, h.data_ptr(), sl.data_ptr(), stream())
            gi.eval_slots_dev(B, h.data_ptr(), sl.data_ptr(), f.data_ptr(), stream())
            gi.select_dev(R, P, g, m.data_ptr(), f.data_ptr(), d_anc.data_ptr(), d_af.data_ptr(),
                          d_best.data_ptr(), d_bf.data_ptr(), stream())
        best = np.flatnonzero(unpack_masks(host(d_best).view(np.uint32)[None], n)[0])
        np.testing.assert_array_equal(fused["hubs"], best)
        assert fused["cost_fp32"] == host(d_bf)[0]


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_solve_tiny_reaches_brute_force_nearest_optimum(path):
    inst = synth.tiny()
    bf = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=1, island_size=64, n1=10, path=path)
        r = gi.solve(100, 2024)
    assert r["cost_fp64"] == pytest.approx(bf["nearest"][0], rel=1e-12)
    assert r["cost_fp64"] >= bf["opt"][0] * (1 - 1e-12)
    cost.check_allocation(inst.n, r["hubs"], r["S"])
    np.testing.assert_array_equal(r["S"], cost.nearest_allocation(inst.C, r["hubs"]))
    assert abs(r["cost_fp32"] - r["cost_fp64"]) / r["cost_fp64"] <= 1e-4
    assert r["evals"] == 1 + 100 * 64


@pytest.mark.parametrize("use_graph", [0, 1])
def test_solve_graph_and_eager_agree(use_graph):
    inst = synth.urand200(seed=33, n=150, p=8)
    out = []
    for ug in (0, 1):
        with Instance.from_instance(inst) as gi:
            gi.set_params(islands=4, island_size=16, n1=5, path=PATH_PLAIN_FP32, use_graph=ug)
            out.append(gi.solve(30, 99))
    np.testing.assert_array_equal(out[0]["hubs"], out[1]["hubs"])
    assert out[0]["cost_fp32"] == out[1]["cost_fp32"]
    assert out[0]["cost_fp64"] == out[1]["cost_fp64"]


def _asym(seed, n, p):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0, 5, (n, n)).astype(np.float32)
    C = rng.uniform(1, 50, (n, n)).astype(np.float32)
    np.fill_diagonal(C, 0)
    return synth.Instance(f"asym{n}", n, p, W, C)


@pytest.mark.parametrize("n,p,B", [(150, 6, 40), (333, 7, 24)])
def test_allocation_bit_exact_asymmetric_c(n, p, B):
    """Nearest allocation compares C[i][hub] (row i), which differs from
    C[hub][i] here: the kernel's transposed reads must pick the oracle's hubs."""
    inst = _asym(n + 3, n, p)
    masks = synth.random_masks(n + 4, n, p, B)
    hubs = np.stack([np.flatnonzero(m) for m in masks]).astype(np.int32)
    with Instance.from_instance(inst) as gi:
        slot = torch.zeros((B, gi.ns), dtype=torch.uint8, device="cuda")
        d_hubs = dev(hubs)
        gi.allocate_dev(B, d_hubs.data_ptr(), slot.data_ptr(), stream())
        got = host(slot)
    for b in range(B):
        ref = cost.slots_of(hubs[b], cost.nearest_allocation(inst.C, hubs[b]))
        np.testing.assert_array_equal(got[b, :n], ref)


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_ga_run_on_asymmetric_c_follows_the_oracle(path):
    """The graph-replayed generation on an asymmetric C (the tensor cores take
    the unfolded W): every generation's children equal the oracle's, their
    fitness is within the path's tolerance of the fp64 objective, and the
    ancestors after selection are the oracle's, fed the GPU's fitness."""
    n, p, R, P, N1, seed, G = 150, 6, 4, 8, 2, 515, 3
    inst = _asym(41, n, p)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path, use_graph=1)
        assert gi.info()["tc_folded"] == 0
        gi.ga_begin(seed)
        am, af = gi.ga_islands()
        st = ga.State(unpack_masks(am, n), af.astype(np.float64), unpack_masks(am, n)[0], float(af[0]))
        for g in range(G):
            gi.ga_run(1)
            masks, fit = gi.ga_population()
            children = ga.make_children(st.ancestors, seed, g, p, P)
            np.testing.assert_array_equal(unpack_masks(masks, n), children)
            _, hh, _ = ga.allocate_all(inst.C, children)
            ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, x) for x in hh])
            assert (np.abs(fit - ref) / ref).max() <= (1e-5 if path == PATH_PLAIN_FP32 else 1e-4)
            ga.select(st, children, fit.astype(np.float64), g, P, N1)
            am, af = gi.ga_islands()
            np.testing.assert_array_equal(unpack_masks(am, n), st.ancestors)
            np.testing.assert_array_equal(af, st.anc_fit.astype(np.float32))


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
@pytest.mark.parametrize("n,p", [(260, 100), (300, 230)])
def test_ga_run_with_large_p_follows_the_oracle(n, p, path):
    """Large p: hub-cost tables too big for the shared slab (p = 100, the
    tensor-core epilogue reads them from global memory) or for the plain
    evaluator's shared table (p = 230); the graph-replayed generations still
    follow the oracle generation by generation."""
    R, P, N1, seed, G = 2, 8, 2, 909, 3
    inst = synth.urand200(seed=n + p, n=n, p=p)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path, use_graph=1)
        gi.ga_begin(seed)
        am, af = gi.ga_islands()
        st = ga.State(unpack_masks(am, n), af.astype(np.float64), unpack_masks(am, n)[0], float(af[0]))
        for g in range(G):
            gi.ga_run(1)
            masks, fit = gi.ga_population()
            children = ga.make_children(st.ancestors, seed, g, p, P)
            np.testing.assert_array_equal(unpack_masks(masks, n), children)
            _, hh, _ = ga.allocate_all(inst.C, children)
            ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, x) for x in hh])
            assert (np.abs(fit - ref) / ref).max() <= (1e-5 if path == PATH_PLAIN_FP32 else 1e-4)
            ga.select(st, children, fit.astype(np.float64), g, P, N1)
            am, af = gi.ga_islands()
            np.testing.assert_array_equal(unpack_masks(am, n), st.ancestors)


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_ga_run_elitist_follows_the_oracle(path):
    """The fused reduction + selection of the replayed generation with the
    elitist flag (an ancestor is kept unless a child is strictly better) and
    merges every second generation: ancestors and their fitness after every
    generation, and the best-ever solution at the end, equal the oracle's."""
    n, p, R, P, N1, seed, G = 120, 6, 3, 8, 2, 6161, 6
    inst = synth.urand200(seed=19, n=n, p=p)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path, elitist=1, use_graph=1)
        gi.ga_begin(seed)
        am, af = gi.ga_islands()
        st = ga.State(unpack_masks(am, n), af.astype(np.float64), unpack_masks(am, n)[0], float(af[0]))
        for g in range(G):
            gi.ga_run(1)
            masks, fit = gi.ga_population()
            children = ga.make_children(st.ancestors, seed, g, p, P)
            np.testing.assert_array_equal(unpack_masks(masks, n), children)
            ga.select(st, children, fit.astype(np.float64), g, P, N1, elitist=True)
            am, af = gi.ga_islands()
            np.testing.assert_array_equal(unpack_masks(am, n), st.ancestors)
            np.testing.assert_array_equal(af, st.anc_fit.astype(np.float32))
        res = gi.ga_result()
    np.testing.assert_array_equal(res["hubs"], np.flatnonzero(st.best))
    assert np.float32(res["cost_fp32"]) == np.float32(st.best_fit)

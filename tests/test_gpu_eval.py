"""GPU evaluation vs the FP64 oracle (objective 1 of §3), through the C ABI."""
import zlib

import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, stream, torch, unpack_masks
from oracle import cost
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance, UsaphmpError

pytestmark = pytest.mark.gpu

# Relative error bounds against the FP64 oracle: fp32 CUDA-core path and
# split-bf16 tensor-core path (W = hi + lo, fp32 accumulation).
TOL = {PATH_PLAIN_FP32: 1e-5, PATH_SPLIT_BF16: 1e-4}
PATHS = [PATH_PLAIN_FP32, PATH_SPLIT_BF16]


def asym_instance(seed, n, p):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0, 5, (n, n)).astype(np.float32)
    C = rng.uniform(1, 50, (n, n)).astype(np.float32)
    np.fill_diagonal(C, 0)
    return synth.Instance(f"asym{n}", n, p, W, C)


def self_flow_instance(seed, n, p):
    """Symmetric C with self-flows W_ii > 0 (the folded operand keeps W_ii on its diagonal)."""
    inst = synth.urand200(seed=seed, n=n, p=p)
    W = inst.W.copy()
    np.fill_diagonal(W, np.random.default_rng(seed).uniform(1, 20, n).astype(np.float32))
    return synth.Instance(f"selfflow{n}", n, p, W, inst.C)


CASES = {
    "tiny_n10_p3": lambda: synth.tiny(),
    "n2_p1": lambda: synth.tiny(seed=5, n=2, p=1),
    "n10_p10": lambda: synth.tiny(seed=6, n=10, p=10),
    "n200_p5": lambda: synth.urand200(p=5),
    "n200_p10": lambda: synth.urand200(p=10),
    "n200_p20": lambda: synth.urand200(p=20),
    "n333_p7_ragged": lambda: synth.urand200(seed=77, n=333, p=7),
    "n257_p1": lambda: synth.urand200(seed=78, n=257, p=1),
    "n129_p64": lambda: synth.urand200(seed=79, n=129, p=64),
    "n140_p50": lambda: synth.urand200(seed=83, n=140, p=50),
    "n300_p63": lambda: synth.urand200(seed=81, n=300, p=63),
    "n260_p100": lambda: synth.urand200(seed=82, n=260, p=100),
    "n240_p226_plain_smem_edge": lambda: synth.urand200(seed=84, n=240, p=226),
    "n300_p255_max": lambda: synth.urand200(seed=85, n=300, p=255),
    "asym_n150_p6": lambda: asym_instance(80, 150, 6),
    "asym_n333_p7_ragged": lambda: asym_instance(86, 333, 7),
    "asym_n300_p63": lambda: asym_instance(87, 300, 63),
    "selfflow_n333_p9": lambda: self_flow_instance(88, 333, 9),
}


def oracle_costs(inst, S):
    return np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s) for s in S])


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_eval_matches_oracle(case, path):
    inst = CASES[case]()
    B = 37
    hubs, S = synth.random_population(zlib.crc32(case.encode()) % 1000, inst.n, inst.p, B)
    ref = oracle_costs(inst, S)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        got = gi.eval(hubs, S)
    rel = np.abs(got - ref) / ref
    assert rel.max() <= TOL[path], (case, rel.max())


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
def test_eval_dev_equals_eval_and_is_repeatable(path):
    inst = synth.urand200(p=10)
    hubs, S = synth.random_population(3, inst.n, inst.p, 300)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        a = gi.eval(hubs, S)
        dh, dS = dev(hubs), dev(S)
        f = torch.empty(300, dtype=torch.float32, device="cuda")
        gi.eval_dev(300, dh.data_ptr(), dS.data_ptr(), f.data_ptr(), stream())
        b = host(f)
        gi.eval_dev(300, dh.data_ptr(), dS.data_ptr(), f.data_ptr(), stream())
        c = host(f)
    np.testing.assert_array_equal(a.astype(np.float32), b)
    np.testing.assert_array_equal(b, c)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
def test_fitness_of_a_chromosome_does_not_depend_on_its_batch(path):
    inst = synth.urand200(seed=9, n=300, p=12)
    hubs, S = synth.random_population(4, inst.n, inst.p, 200)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        whole = gi.eval(hubs, S)
        alone = np.array([gi.eval(hubs[b:b + 1], S[b:b + 1])[0] for b in (0, 1, 57, 199)])
        part = gi.eval(hubs[50:120], S[50:120])
    np.testing.assert_array_equal(whole[[0, 1, 57, 199]], alone)
    np.testing.assert_array_equal(whole[50:120], part)


def test_empty_population():
    inst = synth.tiny()
    with Instance.from_instance(inst) as gi:
        out = gi.eval(np.zeros((0, inst.p), np.int32), np.zeros((0, inst.n), np.int32))
    assert out.shape == (0,)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
@pytest.mark.parametrize("mutate,bad", [
    ("dup_hub", 2), ("spoke_to_nonhub", 5), ("hub_not_self", 1), ("hub_out_of_range", 7), ("S_out_of_range", 3),
])
def test_invalid_chromosomes_are_rejected(mutate, bad, path):
    inst = synth.urand200(seed=11, n=40, p=4)
    hubs, S = synth.random_population(12, inst.n, inst.p, 10)
    h = hubs[bad]
    if mutate == "dup_hub":
        hubs[bad, 1] = hubs[bad, 0]
    elif mutate == "spoke_to_nonhub":
        spoke = next(i for i in range(inst.n) if i not in set(h.tolist()))
        S[bad, spoke] = spoke
    elif mutate == "hub_not_self":
        S[bad, h[0]] = h[1]
    elif mutate == "hub_out_of_range":
        hubs[bad, 2] = inst.n
    elif mutate == "S_out_of_range":
        S[bad, 0] = -1
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        with pytest.raises(UsaphmpError) as e:
            gi.eval(hubs, S)
        assert e.value.name == "EINVAL_CHROM" and f"chromosome {bad}" in str(e.value)
        # the handle stays usable
        good_h, good_S = synth.random_population(13, inst.n, inst.p, 3)
        assert np.isfinite(gi.eval(good_h, good_S)).all()


@pytest.mark.parametrize("what", ["nan_C", "neg_W", "inf_W", "p_gt_n", "p0", "n1"])
def test_create_rejects_bad_instances(what):
    inst = synth.tiny()
    W, C, p, n = inst.W.copy(), inst.C.copy(), inst.p, inst.n
    if what == "nan_C":
        C[2, 3] = np.nan
    elif what == "neg_W":
        W[1, 4] = -1
    elif what == "inf_W":
        W[0, 9] = np.inf
    elif what == "p_gt_n":
        p = n + 1
    elif what == "p0":
        p = 0
    elif what == "n1":
        W, C, p = W[:1, :1], C[:1, :1], 1
    with pytest.raises(UsaphmpError) as e:
        Instance(W, C, p)
    assert e.value.name == "EINVAL"


def test_rescore_fp64_matches_oracle():
    inst = synth.urand200(seed=21, n=300, p=9)
    hubs, S = synth.random_population(22, inst.n, inst.p, 6)
    ref = oracle_costs(inst, S)
    with Instance.from_instance(inst) as gi:
        hs = np.sort(hubs, axis=1).astype(np.int32)
        slot = np.full((6, gi.ns), 255, np.uint8)
        for b in range(6):
            slot[b, :inst.n] = cost.slots_of(hs[b], S[b])
        c = torch.empty(6, dtype=torch.float64, device="cuda")
        d_hs, d_slot = dev(hs), dev(slot)   # keep the tensors alive while the kernels run
        gi.rescore_fp64_dev(6, d_hs.data_ptr(), d_slot.data_ptr(), c.data_ptr(), stream())
        got = host(c)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
@pytest.mark.parametrize("B", [511, 512, 2047, 2500, 4099, 8800])
def test_host_eval_in_chunks_equals_device_eval(path, B):
    """usaphmp_eval copies and evaluates large populations in chunks; the
    fitness equals the single-launch device call bit for bit."""
    inst = synth.urand200(seed=31, n=150, p=9)
    hubs, S = synth.random_population(32, inst.n, inst.p, B)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=path)
        got = gi.eval(hubs, S)
        f = torch.empty(B, dtype=torch.float32, device="cuda")
        d_h, d_S = dev(hubs), dev(S)
        gi.eval_dev(B, d_h.data_ptr(), d_S.data_ptr(), f.data_ptr(), stream())
        ref_dev = host(f).astype(np.float64)
    np.testing.assert_array_equal(got, ref_dev)
    idx = np.array([0, B // 3, B // 2, B - 1])
    ref = oracle_costs(inst, S[idx])
    assert (np.abs(got[idx] - ref) / ref).max() <= TOL[path]


def test_host_eval_reports_a_bad_chromosome_in_a_later_chunk():
    inst = synth.urand200(seed=33, n=60, p=5)
    B, bad = 2100, 1800
    hubs, S = synth.random_population(34, inst.n, inst.p, B)
    hubs[bad, 1] = hubs[bad, 0]
    with Instance.from_instance(inst) as gi:
        with pytest.raises(UsaphmpError) as e:
            gi.eval(hubs, S)
        assert e.value.name == "EINVAL_CHROM" and f"chromosome {bad}" in str(e.value)
        hubs[bad] = hubs[bad - 1]
        S[bad] = S[bad - 1]
        out = gi.eval(hubs, S)
        assert out[bad] == out[bad - 1]


def test_misaligned_slot_buffers_are_refused():
    inst = synth.urand200(seed=35, n=40, p=4)
    with Instance.from_instance(inst) as gi:
        hubs = torch.zeros((2, inst.p), dtype=torch.int32, device="cuda")
        raw = torch.zeros(2 * gi.ns + 4, dtype=torch.uint8, device="cuda")
        fit = torch.zeros(2, dtype=torch.float32, device="cuda")
        for call in (lambda: gi.allocate_dev(2, hubs.data_ptr(), raw.data_ptr() + 1, stream()),
                     lambda: gi.eval_slots_dev(2, hubs.data_ptr(), raw.data_ptr() + 1, fit.data_ptr(), stream())):
            with pytest.raises(UsaphmpError) as e:
                call()
            assert e.value.name == "EINVAL" and "aligned" in str(e.value)


def test_folded_operand_follows_symmetry():
    """The tensor-core operand is folded exactly when C is symmetric."""
    for inst, folded in ((synth.urand200(seed=90, n=70, p=4), 1), (asym_instance(91, 70, 4), 0)):
        with Instance.from_instance(inst) as gi:
            info = gi.info()
            assert (info["c_symmetric"], info["tc_folded"]) == (folded, folded)
            assert (info["n"], info["p"], info["ns"]) == (inst.n, inst.p, gi.ns)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "split"])
@pytest.mark.parametrize("n,R,P", [(1000, 8, 64), (2500, 4, 32)])
def test_host_eval_of_ga_children_gives_the_ga_fitness(n, R, P, path):
    """The GA's allocation kernel (nearest hub search) and the host-buffer
    evaluation (canonical form of hub ids + S) sum the access terms in the same
    order, so a child of the GA evaluated again through usaphmp_eval, with the
    oracle's nearest allocation as its S, gets the GA's fitness bit for bit
    (one warp per chromosome at n = 1000, two at n = 2500)."""
    inst = synth.clustered(seed=2100 + n, n=n, p=20)
    rng = np.random.default_rng(n)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=5, path=path)
        gi.ga_begin(77)
        gi.ga_run(3)
        masks, fit = gi.ga_population()
        bits = unpack_masks(masks, n)
        idx = np.sort(rng.choice(R * P, 24, replace=False))
        hubs = np.stack([np.flatnonzero(bits[b]) for b in idx]).astype(np.int32)
        S = np.stack([cost.nearest_allocation(inst.C, h) for h in hubs]).astype(np.int32)
        got = gi.eval(hubs[::-1].copy(), S[::-1].copy())[::-1]   # another order and batch
    np.testing.assert_array_equal(got, fit[idx].astype(np.float64))

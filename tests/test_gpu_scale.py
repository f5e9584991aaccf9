"""Output scales of §4.3 (raw, x10^-3, per unit flow), through the C ABI."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, stream, torch
from oracle import cost
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import (PATH_PLAIN_FP32, PATH_SPLIT_BF16, SCALE_MILLI, SCALE_PER_FLOW,
                                            SCALE_RAW, Instance, UsaphmpError)

pytestmark = pytest.mark.gpu

TOL = {PATH_PLAIN_FP32: 1e-5, PATH_SPLIT_BF16: 1e-4}
MODES = {SCALE_RAW: "raw", SCALE_MILLI: "milli", SCALE_PER_FLOW: "per_flow"}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_eval_and_rescore_are_scaled(path):
    inst = synth.urand200(seed=91, n=220, p=9)
    B = 12
    hubs, S = synth.random_population(92, inst.n, inst.p, B)
    raw_ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s) for s in S])
    hs = np.sort(hubs, axis=1).astype(np.int32)
    with Instance.from_instance(inst) as gi:
        slot = np.full((B, gi.ns), 255, np.uint8)
        for b in range(B):
            slot[b, :inst.n] = cost.slots_of(hs[b], S[b])
        d_hs, d_slot = dev(hs), dev(slot)
        gi.set_params(path=path, scale=SCALE_RAW)
        raw = gi.eval(hubs, S)
        for mode, name in MODES.items():
            gi.set_params(scale=mode)
            got = gi.eval(hubs, S)
            ref = np.array([cost.scaled_cost(v, inst.W, name) for v in raw_ref])
            assert (np.abs(got - ref) / ref).max() <= TOL[path]
            factor = ref[0] / raw_ref[0]
            np.testing.assert_allclose(got, raw * factor, rtol=2e-7)     # one fp32 product
            c = torch.empty(B, dtype=torch.float64, device="cuda")
            gi.rescore_fp64_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), c.data_ptr(), stream())
            np.testing.assert_allclose(host(c), ref, rtol=1e-12)


def test_solve_is_the_same_search_under_every_scale():
    inst = synth.urand200(seed=93, n=120, p=6)
    out = {}
    for mode in MODES:
        with Instance.from_instance(inst) as gi:
            gi.set_params(islands=4, island_size=16, n1=5, scale=mode)
            out[mode] = gi.solve(25, 7)
    base = out[SCALE_RAW]
    for mode, name in MODES.items():
        np.testing.assert_array_equal(out[mode]["hubs"], base["hubs"])
        np.testing.assert_array_equal(out[mode]["S"], base["S"])
        assert out[mode]["cost_fp64"] == pytest.approx(cost.scaled_cost(base["cost_fp64"], inst.W, name), rel=1e-14)
        assert out[mode]["cost_fp32"] == pytest.approx(cost.scaled_cost(base["cost_fp32"], inst.W, name), rel=2e-7)


def test_bad_scales_are_refused():
    inst = synth.urand200(seed=94, n=30, p=3)
    with Instance.from_instance(inst) as gi:
        with pytest.raises(UsaphmpError):
            gi.set_params(scale=3)
        assert gi.params["scale"] == SCALE_RAW
    W0 = np.zeros_like(inst.W)
    with Instance(W0, inst.C, inst.p) as gi:
        with pytest.raises(UsaphmpError) as e:
            gi.set_params(scale=SCALE_PER_FLOW)
        assert e.value.name == "EINVAL"
        gi.set_params(scale=SCALE_MILLI)


def _nearest_optimum(inst, chi, alpha, delta):
    """Best nearest-allocation solution over every hub set (oracle)."""
    import itertools
    best = (np.inf, None)
    for hubs in itertools.combinations(range(inst.n), inst.p):
        h = cost.nearest_allocation(inst.C, np.array(hubs))
        c = cost.pair_cost(inst.W, inst.C, chi, alpha, delta, h)
        if c < best[0]:
            best = (c, np.array(hubs))
    return best


@pytest.mark.parametrize("chi_delta,alpha", [(0.5, 0.2), (1.0, 0.6), (3.0, 0.2), (3.0, 1.0)])
def test_factor_sweep_points_reach_the_nearest_optimum(chi_delta, alpha):
    """The chi/delta/alpha study of §6.2 (Fig. 3) at a size the oracle can
    enumerate: each point's GA solution is the best nearest-allocation one."""
    inst = synth.tiny(seed=95, n=10, p=3)
    ref, ref_hubs = _nearest_optimum(inst, chi_delta, alpha, chi_delta)
    with Instance(inst.W, inst.C, inst.p, chi=chi_delta, alpha=alpha, delta=chi_delta) as gi:
        gi.set_params(islands=2, island_size=64, n1=10, scale=SCALE_PER_FLOW)
        r = gi.solve(100, 11)
    assert r["cost_fp64"] == pytest.approx(cost.scaled_cost(ref, inst.W, "per_flow"), rel=1e-12)
    np.testing.assert_array_equal(np.sort(r["hubs"]), ref_hubs)

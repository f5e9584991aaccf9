"""The allocation-free fp64 rescoring entry point, through the C ABI.

usaphmp_rescore_fp64_noalloc serves callers that cannot call cudaMalloc (a
fixed device-memory budget or pool owned by the host application, or a loop
that cannot take cudaMalloc's implicit synchronisation): it takes only caller
buffers and keeps its partial sums in a fixed scratch array inside the
library.  Its costs must match the oracle's fp64 pair-form objective and
usaphmp_rescore_fp64_dev, the handle-based entry point, on consecutive calls
(the second call reuses the scratch the first one left behind), for a
symmetric and an asymmetric C.
"""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu, stream, torch
from oracle import cost as ocost
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import Instance, UsaphmpError, rescore_fp64_noalloc

pytestmark = pytest.mark.gpu

RTOL = 1e-12   # fp64 rescoring, same tolerance as the other fp64 tests


def _canonical(inst, hubs, S, stride):
    hs = np.sort(hubs, axis=1).astype(np.int32)
    slot = np.full((hubs.shape[0], stride), 255, np.uint8)
    for b in range(hubs.shape[0]):
        slot[b, :inst.n] = ocost.slots_of(hs[b], S[b])
    return hs, slot


def _asymmetric(inst, seed):
    """The same instance with C made asymmetric (each arc's cost scaled by its
    own factor in [0.8, 1.25], diagonal kept at 0)."""
    rng = np.random.default_rng(seed)
    C = (inst.C * rng.uniform(0.8, 1.25, inst.C.shape)).astype(np.float32)
    np.fill_diagonal(C, 0.0)
    assert not np.array_equal(C, C.T)
    return synth.Instance(inst.name + "-asym", inst.n, inst.p, inst.W, C)


@pytest.mark.parametrize("sym", [True, False], ids=["symmetric_C", "asymmetric_C"])
def test_noalloc_rescore_matches_the_oracle_and_the_handle_entry_point_on_two_calls(sym):
    need_gpu()
    inst = synth.urand200(seed=91, n=333, p=9)
    if not sym:
        inst = _asymmetric(inst, 94)
    W_d, C_d = dev(inst.W), dev(inst.C)
    with Instance.from_instance(inst) as gi:
        assert gi.info()["c_symmetric"] == int(sym)
        for call, B in enumerate((12, 37)):
            hubs, S = synth.random_population(92 + call, inst.n, inst.p, B)
            hs, slot_pad = _canonical(inst, hubs, S, gi.ns)
            _, slot_dense = _canonical(inst, hubs, S, inst.n)
            d_hs, d_pad, d_dense = dev(hs), dev(slot_pad), dev(slot_dense)
            ref = torch.empty(B, dtype=torch.float64, device="cuda")
            got = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
            gi.rescore_fp64_dev(B, d_hs.data_ptr(), d_pad.data_ptr(), ref.data_ptr(), stream())
            rescore_fp64_noalloc(inst.n, inst.p, B, W_d.data_ptr(), C_d.data_ptr(), inst.chi, inst.alpha,
                                 inst.delta, d_hs.data_ptr(), d_dense.data_ptr(), got.data_ptr(), stream())
            got_h = host(got)
            np.testing.assert_allclose(got_h, host(ref), rtol=RTOL)
            oracle = np.array([ocost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, S[b])
                               for b in range(B)])
            np.testing.assert_allclose(got_h, oracle, rtol=RTOL)


def test_noalloc_rescore_rejects_sizes_beyond_its_scratch():
    need_gpu()
    inst = synth.urand200(seed=93, n=300, p=5)
    W_d, C_d = dev(inst.W), dev(inst.C)
    B = 131072 // 128 + 1
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    hubs = torch.zeros((B, inst.p), dtype=torch.int32, device="cuda")
    slot = torch.zeros((B, inst.n), dtype=torch.uint8, device="cuda")
    with pytest.raises(UsaphmpError) as e:
        rescore_fp64_noalloc(inst.n, inst.p, B, W_d.data_ptr(), C_d.data_ptr(), inst.chi, inst.alpha, inst.delta,
                             hubs.data_ptr(), slot.data_ptr(), out.data_ptr(), stream())
    assert e.value.name == "EINVAL" and "scratch" in str(e.value)

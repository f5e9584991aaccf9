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

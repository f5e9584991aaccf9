"""Tile shapes of the tensor-core evaluator and the autotuner, through the C ABI."""
import json

import numpy as np
import pytest

from gpu_util import need_gpu
from oracle import cost
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance, UsaphmpError

pytestmark = pytest.mark.gpu

# (ntile, stages, raster, pair): one CTA per MMA (ntile 256: at most 3 stages),
# or CTA pairs with M = 256 MMAs (half the one-hot operand per CTA: 4 stages fit)
SHAPES = [(nt, st, ra, 0) for nt in (256, 128, 64) for st in (2, 3, 4) for ra in (0, 1) if not (nt == 256 and st == 4)]
SHAPES += [(nt, st, ra, 1) for nt in (256, 128, 64) for st in (2, 3, 4) for ra in (0, 1)]
KEYS = ("ntile", "stages", "raster", "pair")
DEFAULT = {"ntile": 256, "stages": 3, "raster": 0, "pair": 0}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("n,p,B", [(333, 7, 91), (200, 20, 64), (129, 64, 10), (1000, 20, 300)])
def test_every_shape_gives_bit_identical_fitness(n, p, B):
    inst = synth.urand200(seed=n + p, n=n, p=p)
    hubs, S = synth.random_population(n * 7 + p, n, p, B)
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=PATH_SPLIT_BF16)
        assert gi.get_tile() == DEFAULT
        base = gi.eval(hubs, S)
        for shape in SHAPES:
            if shape[0] < p:
                with pytest.raises(UsaphmpError):
                    gi.set_tile(*shape)
                continue
            gi.set_tile(*shape)
            assert gi.get_tile() == dict(zip(KEYS, shape))
            np.testing.assert_array_equal(gi.eval(hubs, S), base, err_msg=str(shape))
    ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s) for s in S[:8]])
    assert (np.abs(base[:8] - ref) / ref).max() <= 1e-4


@pytest.mark.parametrize("shape", [(32, 3, 0), (512, 2, 0), (256, 4, 0), (128, 1, 0), (128, 5, 0), (128, 3, 2),
                                   (128, 3, 0, 2), (256, 5, 0, 1), (64, 3, 0)])
def test_invalid_shapes_are_refused(shape):
    inst = synth.urand200(seed=3, n=120, p=100)
    with Instance.from_instance(inst) as gi:
        with pytest.raises(UsaphmpError) as e:
            gi.set_tile(*shape)           # the last one: ntile 64 < p = 100
        assert e.value.name == "EINVAL"
        assert gi.get_tile() == DEFAULT


def test_autotune_picks_a_valid_shape_and_caches_it(tmp_path):
    inst = synth.urand200(seed=12, n=300, p=10)
    cache = str(tmp_path / "tiles.json")
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=4, island_size=32, path=PATH_SPLIT_BF16)
        got = gi.autotune(reps=3, cache=cache)
        assert tuple(got[k] for k in KEYS) in SHAPES
        assert not got["from_cache"]
        assert 0 < got["ms"] <= got["default_ms"]
        assert gi.get_tile() == {k: got[k] for k in KEYS}
        with pytest.raises(UsaphmpError):
            gi.ga_run(1)                   # the tuner reset the GA state
        entries = json.load(open(cache))["entries"]
        assert len(entries) == 1 and entries[0]["p"] == 10 and entries[0]["n_blocks"] == 3
        assert entries[0]["B_pow2"] == 128
        tuned = gi.solve(generations=12, seed=5)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=4, island_size=32, path=PATH_SPLIT_BF16)
        again = gi.autotune(reps=3, cache=cache)
        assert again["from_cache"] and again["ms"] == 0.0
        assert {k: again[k] for k in KEYS} == {k: got[k] for k in KEYS}
        gi.set_tile(256, 3, 0)
        default = gi.solve(generations=12, seed=5)
    # the shape changes speed only
    assert tuned["cost_fp64"] == default["cost_fp64"] and tuned["cost_fp32"] == default["cost_fp32"]
    np.testing.assert_array_equal(tuned["hubs"], default["hubs"])


def test_autotune_on_the_plain_path_keeps_the_shape(tmp_path):
    inst = synth.urand200(seed=13, n=150, p=6)
    cache = str(tmp_path / "tiles.json")
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=PATH_PLAIN_FP32)
        got = gi.autotune(reps=2, cache=cache)
        assert {k: got[k] for k in ("ntile", "stages", "raster")} == {"ntile": 256, "stages": 3, "raster": 0}
        assert got["ms"] == 0.0 and not got["from_cache"]
    assert not (tmp_path / "tiles.json").exists()


def test_cache_buckets_separate_folded_and_full_operands(tmp_path):
    """A shape tuned on a symmetric instance (folded operand) is not reused for
    an asymmetric instance of the same size, and the reverse."""
    cache = str(tmp_path / "tiles.json")
    sym = synth.urand200(seed=17, n=260, p=9)
    C = sym.C.copy()
    C[0, 1] += 1.0          # one asymmetric pair: the full W operand
    asym = synth.Instance("asym260", sym.n, sym.p, sym.W, C)
    for inst in (sym, asym):
        with Instance.from_instance(inst) as gi:
            gi.set_params(islands=4, island_size=32, path=PATH_SPLIT_BF16)
            got = gi.autotune(reps=2, cache=cache)
            assert not got["from_cache"]
    devices = sorted(e["device"] for e in json.load(open(cache))["entries"])
    assert len(devices) == 2 and devices[1] == devices[0] + " (folded operand)"

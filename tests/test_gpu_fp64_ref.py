"""The fp64 reference evaluator path (USAPHMP_PATH_FP64_REF): fitness equal to
the oracle's cost rounded to fp32, and a whole GA run that makes the oracle's
decisions."""
import numpy as np
import pytest

from gpu_util import need_gpu
from oracle import brute, cost, ga
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_FP64_REF, ROUTE_HUB_PATHS, Instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("routing", ["direct", "hubs"])
def test_fp64_path_fitness_is_the_rounded_oracle_cost(routing):
    inst = synth.latency_like(seed=101, n=230, p=11)
    hubs, S = synth.random_population(102, inst.n, inst.p, 23)
    ref = np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s, routing) for s in S])
    with Instance.from_instance(inst) as gi:
        gi.set_params(path=PATH_FP64_REF, routing=ROUTE_HUB_PATHS if routing == "hubs" else 0)
        got = gi.eval(hubs, S)
    np.testing.assert_allclose(got, ref.astype(np.float32).astype(np.float64), rtol=1.2e-7)


@pytest.mark.parametrize("seed", [3, 4])
def test_fp64_path_ga_follows_the_oracle_ga(seed):
    inst = synth.urand200(seed=103 + seed, n=36, p=4)
    R, P, N1, G = 2, 16, 4, 14
    hubs_o, h_o, cost_o, st = ga.solve(inst, generations=G, seed=seed, R=R, P=P, N1=N1)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=PATH_FP64_REF)
        r = gi.solve(G, seed)
    np.testing.assert_array_equal(np.sort(r["hubs"]), np.sort(hubs_o))
    np.testing.assert_array_equal(r["S"], h_o)
    assert r["cost_fp64"] == pytest.approx(cost_o, rel=1e-12)


def test_fp64_path_solve_reaches_the_brute_force_nearest_optimum():
    inst = synth.tiny()
    bf = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=1, island_size=64, n1=10, path=PATH_FP64_REF)
        r = gi.solve(100, 2024)
    assert r["cost_fp64"] == pytest.approx(bf["nearest"][0], rel=1e-12)
    assert r["cost_fp32"] == np.float32(r["cost_fp64"])


@pytest.mark.parametrize("path", [0, 1], ids=["plain", "split"])
@pytest.mark.parametrize("seed", [3, 6])
def test_fast_paths_ga_follows_the_oracle_ga_when_decisions_have_margin(path, seed):
    """On these runs every selection, merge and best-ever comparison of the
    oracle GA is decided by a relative margin of at least 4.7e-4 (checked on
    the oracle side), far above the fp32 / split-bf16 fitness error, so the
    fast paths must make the same decisions."""
    inst = synth.urand200(seed=103 + seed, n=36, p=4)
    R, P, N1, G = 2, 16, 4, 14
    hubs_o, h_o, cost_o, _ = ga.solve(inst, generations=G, seed=seed, R=R, P=P, N1=N1)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=R, island_size=P, n1=N1, path=path)
        r = gi.solve(G, seed)
    np.testing.assert_array_equal(np.sort(r["hubs"]), np.sort(hubs_o))
    np.testing.assert_array_equal(r["S"], h_o)
    assert r["cost_fp64"] == pytest.approx(cost_o, rel=1e-12)

"""Pins of the oracle's allocation local search."""
import os

import numpy as np
import pytest

from oracle import brute, cost
from oracle.local_search import local_search
from paper_1704_06258_gb300 import synth


def _ints(s):
    return np.array([int(v) for v in s.split(",")])


def _hand(golden_dir):
    rows = [ln.split() for ln in open(os.path.join(golden_dir, "hand4_local_search.txt"))
            if ln.strip() and not ln.startswith("#")]
    x = np.array([float(v) for v in next(r for r in rows if r[0] == "x")[1:]])
    W = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "W"], dtype=np.float32)
    chi, alpha, delta = (float(v) for v in next(r for r in rows if r[0] == "params")[1:])
    hubs = _ints(next(r for r in rows if r[0] == "hubs")[1])
    C = np.abs(x[:, None] - x[None, :]).astype(np.float32)
    return rows, W, C, chi, alpha, delta, hubs


def test_hand_worked_search(golden_dir):
    rows, W, C, chi, alpha, delta, hubs = _hand(golden_dir)
    for r in rows:
        if r[0] == "alloc":
            assert cost.pair_cost(W, C, chi, alpha, delta, _ints(r[1])) == pytest.approx(float(r[2]), rel=1e-15)
        if r[0] == "search":
            start = _ints(r[1])
            np.testing.assert_array_equal(start, cost.nearest_allocation(C, hubs))
            h, sweeps, moves = local_search(W, C, chi, alpha, delta, hubs, start, 10)
            np.testing.assert_array_equal(h, _ints(r[2]))
            assert cost.pair_cost(W, C, chi, alpha, delta, h) == pytest.approx(float(r[3]), rel=1e-15)
            assert (sweeps, moves) == (int(r[4]), int(r[5]))


def _heavy_tailed(seed, n, p, spread=0.0):
    inst = synth.latency_like(seed=seed, n=n, p=p, spread=spread)
    rng = np.random.default_rng(seed)
    W = (inst.W * rng.lognormal(0.0, 1.5, size=inst.W.shape)).astype(np.float32)
    np.fill_diagonal(W, 0.0)
    return W, inst.C


def _single_moves(W, C, hubs, h, routing):
    """Cost change of every single reallocation of a spoke (exhaustive)."""
    base = cost.pair_cost(W, C, 3.0, 0.75, 2.0, h, routing)
    out = []
    for i in range(len(h)):
        if i in set(hubs.tolist()):
            continue
        for b in hubs:
            if b != h[i]:
                h2 = h.copy()
                h2[i] = b
                out.append(cost.pair_cost(W, C, 3.0, 0.75, 2.0, h2, routing) - base)
    return np.array(out)


@pytest.mark.parametrize("seed,routing", [(5, "direct"), (9, "direct"), (25, "direct"), (41, "hubs"), (42, "hubs")])
def test_result_is_a_local_optimum_and_never_worse(seed, routing):
    W, C = _heavy_tailed(seed, 12, 3, spread=0.8 if routing == "hubs" else 0.0)
    rng = np.random.default_rng(seed)
    hubs = np.sort(rng.choice(12, 3, replace=False))
    for start in (cost.nearest_allocation(C, hubs), hubs[rng.integers(0, 3, size=12)]):
        start = start.copy()
        start[hubs] = hubs
        h, sweeps, moves = local_search(W, C, 3.0, 0.75, 2.0, hubs, start, 50, routing)
        cost.check_allocation(12, hubs, h)
        assert sweeps < 50
        assert (_single_moves(W, C, hubs, h, routing) >= -1e-9 * cost.pair_cost(W, C, 3, .75, 2, h, routing)).all()
        assert cost.pair_cost(W, C, 3, .75, 2, h, routing) <= cost.pair_cost(W, C, 3, .75, 2, start, routing)
        assert (moves == 0) == (h == start).all()


def test_brute_force_optimum_is_a_fixed_point_and_search_can_reach_it():
    reached = 0
    for seed in (5, 7, 9, 11, 21):
        W, C = _heavy_tailed(seed, 8, 3)
        bf = brute.brute_force(W, C, 3.0, 0.75, 2.0, 3)
        _, hubs, hopt = bf["opt"]
        h, sweeps, moves = local_search(W, C, 3.0, 0.75, 2.0, hubs, hopt, 10)
        assert moves == 0 and sweeps == 1
        h2, _, moves2 = local_search(W, C, 3.0, 0.75, 2.0, hubs, cost.nearest_allocation(C, hubs), 10)
        c2 = cost.pair_cost(W, C, 3.0, 0.75, 2.0, h2)
        assert c2 >= bf["opt"][0] * (1 - 1e-12)
        reached += moves2 > 0 and c2 == pytest.approx(bf["opt"][0], rel=1e-12)
    assert reached >= 3      # nearest allocation was not optimal and the search closed the gap

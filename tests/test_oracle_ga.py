"""Pins of the oracle's random numbers and GA operators."""
import os

import numpy as np
import pytest

from oracle import brute, cost, ga
from oracle.philox import DrawStream, philox4x32_10
from paper_1704_06258_gb300 import synth


def test_philox_known_answers(golden_dir):
    for ln in open(os.path.join(golden_dir, "philox4x32_10_kat.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        w = [int(v, 16) for v in ln.split()]
        assert philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])


def test_draws_uniform_chi_square():
    m = 7
    counts = np.zeros(m)
    for q in range(3000):
        s = DrawStream(12345, 3, q, 1)
        for _ in range(4):
            counts[s.below(m)] += 1
    expect = counts.sum() / m
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 22.5            # 6 d.o.f., p ~ 0.001


class Scripted:
    """A draw stream returning given values of below(m) (checked against m)."""

    def __init__(self, values):
        self.values = list(values)

    def below(self, m):
        v = self.values.pop(0)
        assert 0 <= v < max(m, 1)
        return v


def test_exchange_every_choice():
    base = np.array([0, 1, 1, 0, 0, 1, 0], dtype=bool)
    opened = np.flatnonzero(base)
    closed = np.flatnonzero(~base)
    seen = set()
    for i in range(len(opened)):
        for j in range(len(closed)):
            m = ga.exchange(base.copy(), Scripted([i, j]))
            diff = np.flatnonzero(m != base)
            assert sorted(diff) == sorted([opened[i], closed[j]])
            assert m.sum() == base.sum() and not m[opened[i]] and m[closed[j]]
            seen.add(tuple(m))
    assert len(seen) == len(opened) * len(closed)


def test_exchange_degenerate_masks_consume_two_words():
    for mask in (np.zeros(5, bool), np.ones(5, bool)):
        s = DrawStream(1, 0, 0, 0)
        out = ga.exchange(mask.copy(), s)
        np.testing.assert_array_equal(out, mask)
        assert s.block == 1 and len(s.buf) == 2


def test_crossover_every_cut():
    n = 9
    pa = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1], dtype=bool)
    pb = np.array([0, 1, 0, 0, 1, 1, 0, 1, 0], dtype=bool)   # complement: children show the cut
    for c in range(1, n):
        ca, cb, cut = ga.crossover(pa, pb, Scripted([c - 1]))
        assert cut == c
        np.testing.assert_array_equal(ca, np.r_[pa[:c], pb[c:]])
        np.testing.assert_array_equal(cb, np.r_[pb[:c], pa[c:]])
        assert (ca ^ cb).all()


@pytest.mark.parametrize("h0", [0, 1, 3, 6, 9])
def test_correction_reaches_p(h0):
    n, p = 9, 3
    rng = np.random.default_rng(h0)
    for trial in range(20):
        m = np.zeros(n, bool)
        m[rng.choice(n, h0, replace=False)] = True
        before = m.copy()
        ga.correct(m, p, DrawStream(7, trial, h0, 2))
        assert m.sum() == p
        if h0 >= p:
            assert not (m & ~before).any()       # only closes
        else:
            assert not (~m & before).any()       # only opens


def test_children_are_valid_and_deterministic():
    inst = synth.urand200(seed=51, n=50, p=5)
    anc = synth.random_masks(52, inst.n, inst.p, 3)
    a = ga.make_children(anc, seed=99, g=4, p=inst.p, P=8)
    b = ga.make_children(anc, seed=99, g=4, p=inst.p, P=8)
    c = ga.make_children(anc, seed=99, g=5, p=inst.p, P=8)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()
    assert a.shape == (24, 50) and (a.sum(1) == inst.p).all()
    hubs, h, slot = ga.allocate_all(inst.C, a)
    for q in range(a.shape[0]):
        cost.check_allocation(inst.n, hubs[q], h[q])
        for i in range(inst.n):
            assert inst.C[i, h[q, i]] == inst.C[i, hubs[q]].min() or h[q, i] == i


def test_selection_rules():
    n, P = 6, 4
    anc = np.zeros((2, n), bool)
    children = np.eye(8, n, dtype=bool)
    st = ga.State(anc, [10.0, 10.0], anc[0], 10.0)
    fit = np.array([5.0, 3.0, 3.0, 9.0, 4.0, 2.0, 8.0, 2.0])
    ga.select(st, children, fit, g=0, P=P, N1=10)
    np.testing.assert_array_equal(st.ancestors[0], children[1])   # first of the tied minima
    np.testing.assert_array_equal(st.ancestors[1], children[5])
    assert st.best_fit == 2.0 and (st.best == children[5]).all()
    # merge at the end of an outer iteration
    ga.select(st, children, fit, g=9, P=P, N1=10)
    np.testing.assert_array_equal(st.ancestors[0], children[5])
    # best-ever replaced only on a strict improvement
    fit2 = fit + 1.0
    ga.select(st, children, fit2, g=1, P=P, N1=10)
    assert st.best_fit == 2.0
    # unconditional ancestor replacement (default) vs elitist
    np.testing.assert_array_equal(st.ancestors[1], children[5])
    assert st.anc_fit[1] == 3.0
    st2 = ga.State(children[[1, 5]], [2.5, 1.0], children[5], 1.0)
    ga.select(st2, children, fit, g=1, P=P, N1=10, elitist=True)
    np.testing.assert_array_equal(st2.ancestors[0], children[1])
    assert st2.anc_fit[1] == 1.0


def test_selection_ranks_nan_last():
    n, P = 6, 4
    children = np.eye(8, n, dtype=bool)
    st = ga.State(np.zeros((2, n), bool), [10.0, 10.0], np.zeros(n, bool), 10.0)
    fit = np.array([np.nan, 3.0, np.nan, 5.0, np.nan, np.nan, np.nan, np.nan])
    ga.select(st, children, fit, g=0, P=P, N1=10)
    np.testing.assert_array_equal(st.ancestors[0], children[1])   # NaN never preferred
    np.testing.assert_array_equal(st.ancestors[1], children[4])   # all NaN: first member
    assert st.anc_fit[1] == np.inf and st.best_fit == 3.0


@pytest.mark.slow
def test_ga_reaches_best_nearest_solution_on_tiny_instance():
    inst = synth.tiny()
    bf = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p)
    hubs, h, c, _ = ga.solve(inst, generations=100, seed=2024, R=1, P=64, N1=10)
    assert c >= bf["opt"][0] * (1 - 1e-12)
    assert c == pytest.approx(bf["nearest"][0], rel=1e-12)


def test_sharded_islands_make_the_single_population_decisions():
    """Two shards of two islands each, drawing by global chromosome index and
    merged across shards every N1 generations, follow the run of one
    population of four islands exactly."""
    inst = synth.urand200(seed=53, n=30, p=4)
    seed, P, N1, G = 77, 8, 3, 10

    def fitness(children):
        _, h, _ = ga.allocate_all(inst.C, children)
        return np.array([cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, x) for x in h])

    hubs0, h0 = cost.initial_solution(inst.C, inst.p)
    mask0 = np.zeros(inst.n, dtype=bool)
    mask0[hubs0] = True
    f0 = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, h0)
    whole = ga.State(np.tile(mask0, (4, 1)), np.full(4, f0), mask0, f0)
    shards = [ga.State(np.tile(mask0, (2, 1)), np.full(2, f0), mask0, f0) for _ in range(2)]
    for g in range(G):
        children = ga.make_children(whole.ancestors, seed, g, inst.p, P)
        ga.select(whole, children, fitness(children), g, P, N1)
        for k, st in enumerate(shards):
            ch = ga.make_children(st.ancestors, seed, g, inst.p, P, island_offset=2 * k)
            np.testing.assert_array_equal(ch, children[16 * k:16 * (k + 1)])
            ga.select(st, ch, fitness(ch), g, P, 0)
        if (g + 1) % N1 == 0:
            ga.merge_shards(shards, [2, 2])
        np.testing.assert_array_equal(np.concatenate([s.ancestors for s in shards]), whole.ancestors)
        np.testing.assert_array_equal(np.concatenate([s.anc_fit for s in shards]), whole.anc_fit)
    assert min(s.best_fit for s in shards) == whole.best_fit

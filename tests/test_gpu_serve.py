"""Serving loop: continuous batching, admission, alone-vs-mix determinism."""
import numpy as np
import pytest

from gpu_util import need_gpu
from oracle import cost
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance, Server, UsaphmpError

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _requests():
    out = []
    for r, (n, p, gens) in enumerate([(60, 3, 12), (250, 11, 9), (97, 7, 15), (400, 20, 6), (33, 5, 10)]):
        inst = synth.clustered(seed=7000 + r, n=n, p=p)
        out.append((inst, gens, 100 + r))
    return out


def _drain(server, tickets):
    res = {}
    for _ in range(10000):
        server.step()
        for t in list(tickets):
            r = server.poll(t)
            if r is not None:
                res[t] = r
                tickets.remove(t)
        if not tickets:
            return res
    raise AssertionError("server did not finish")


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_results_alone_equal_results_in_the_mix(path):
    reqs = _requests()
    alone = []
    for inst, gens, seed in reqs:
        with Server(4 * GB, max_active=8, path=path) as s:
            t = s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=gens, seed=seed)
            alone.append(_drain(s, [t])[t])
    with Server(4 * GB, max_active=3, path=path) as s:
        tickets = []
        # staggered arrivals: two now, the rest while those run
        for k, (inst, gens, seed) in enumerate(reqs):
            tickets.append(s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=gens, seed=seed))
            if k >= 1:
                s.step()
        mixed = _drain(s, list(tickets))
    for (inst, gens, seed), a, t in zip(reqs, alone, tickets):
        m = mixed[t]
        np.testing.assert_array_equal(a["hubs"], m["hubs"])
        np.testing.assert_array_equal(a["S"], m["S"])
        assert a["cost_fp32"] == m["cost_fp32"] and a["cost_fp64"] == m["cost_fp64"]
        assert m["evals"] == 1 + gens * 32
        cost.check_allocation(inst.n, m["hubs"], m["S"])
        ref = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, m["S"])
        assert m["cost_fp64"] == pytest.approx(ref, rel=1e-12)


def test_served_result_equals_direct_solve():
    inst = synth.clustered(seed=7100, n=180, p=9)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=2, island_size=16, n1=10, path=PATH_SPLIT_BF16)
        direct = gi.solve(11, 5)
    with Server(4 * GB, max_active=4, path=PATH_SPLIT_BF16) as s:
        t = s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=11, seed=5)
        served = _drain(s, [t])[t]
    np.testing.assert_array_equal(direct["hubs"], served["hubs"])
    assert direct["cost_fp32"] == served["cost_fp32"]


def test_admission_respects_the_memory_budget_and_slots():
    reqs = _requests()
    fp = [Server.footprint(i.n, i.p, 2, 16) for i, _, _ in reqs]
    budget = max(fp) + min(fp)          # never room for the two largest at once
    with Server(budget, max_active=2, path=PATH_SPLIT_BF16) as s:
        tickets = [s.submit(i.W, i.C, i.p, islands=2, island_size=16, generations=g, seed=sd) for i, g, sd in reqs]
        peak = 0
        done = {}
        for _ in range(10000):
            active, pending = s.step()
            peak = max(peak, active)
            for t in list(tickets):
                r = s.poll(t)
                if r is not None:
                    done[t] = r
                    tickets.remove(t)
            if not tickets:
                break
        assert not tickets and peak <= 2


def test_oversized_request_is_refused():
    inst = synth.clustered(seed=7200, n=300, p=5)
    with Server(1 << 20, max_active=2) as s:
        t = s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=3)
        s.step()
        with pytest.raises(UsaphmpError) as e:
            s.poll(t)
        assert e.value.name == "EBUSY"


def test_invalid_request_fails_alone():
    good = synth.clustered(seed=7300, n=80, p=4)
    bad_W = good.W.copy()
    bad_W[3, 4] = -1.0
    with Server(4 * GB, max_active=4) as s:
        tb = s.submit(bad_W, good.C, good.p, islands=2, island_size=16, generations=3)
        tg = s.submit(good.W, good.C, good.p, islands=2, island_size=16, generations=3)
        res = {}
        for _ in range(100):
            s.step()
            for t in (tb, tg):
                if t in res:
                    continue
                try:
                    r = s.poll(t)
                except UsaphmpError as e:
                    r = e
                if r is not None:
                    res[t] = r
            if len(res) == 2:
                break
        assert isinstance(res[tb], UsaphmpError) and res[tb].name == "EINVAL"
        assert isinstance(res[tg], dict)


def test_serving_workload_alone_equals_the_poisson_mix():
    """The serving workload's own requests (n log-uniform in [50, 3000], p in
    3..20, clustered instances seeded 5000 + r, population 512 = 8 x 64, 200
    generations): 16 of them each run alone, then the same 16 inside a mix of
    64 with Poisson arrivals (submitted between steps in arrival order) and up
    to 64 running at once.  Hubs, allocation and both costs are bit-identical,
    and every fp64 cost is the oracle's pair-form objective."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor

    total, checked, gens, R, P = 64, 16, 200, 8, 64
    with ProcessPoolExecutor(min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        reqs = list(ex.map(synth.serving_request, range(total)))
    assert max(r.n for r in reqs[:checked]) > 1000
    alone = []
    for r in range(checked):
        inst = reqs[r]
        with Server(32 * GB, max_active=64, path=PATH_SPLIT_BF16) as s:
            t = s.submit(inst.W, inst.C, inst.p, islands=R, island_size=P, generations=gens, seed=5000 + r)
            alone.append(_drain(s, [t])[t])
    # arrivals: 64 requests over about 40 ticks
    arrival_tick = np.floor(np.cumsum(np.random.default_rng(77).exponential(40.0 / total, total))).astype(int)
    mixed, tickets, nxt, peak = {}, {}, 0, 0
    with Server(32 * GB, max_active=64, path=PATH_SPLIT_BF16) as s:
        for tick in range(100000):
            while nxt < total and arrival_tick[nxt] <= tick:
                inst = reqs[nxt]
                tickets[s.submit(inst.W, inst.C, inst.p, islands=R, island_size=P, generations=gens,
                                 seed=5000 + nxt)] = nxt
                nxt += 1
            active, _ = s.step()
            peak = max(peak, active)
            for t in [t for t in tickets if tickets[t] not in mixed]:
                res = s.poll(t)
                if res is not None:
                    mixed[tickets[t]] = res
            if len(mixed) == total:
                break
    assert len(mixed) == total and peak > 8
    for r in range(checked):
        inst, a, m = reqs[r], alone[r], mixed[r]
        np.testing.assert_array_equal(a["hubs"], m["hubs"])
        np.testing.assert_array_equal(a["S"], m["S"])
        assert a["cost_fp32"] == m["cost_fp32"] and a["cost_fp64"] == m["cost_fp64"]
        assert m["evals"] == 1 + gens * R * P
        cost.check_allocation(inst.n, m["hubs"], m["S"])
        ref = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, m["S"])
        assert m["cost_fp64"] == pytest.approx(ref, rel=1e-12)


def _asym(seed, n, p):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0, 5, (n, n)).astype(np.float32)
    C = rng.uniform(1, 50, (n, n)).astype(np.float32)
    np.fill_diagonal(C, 0)
    return synth.Instance(f"asym{n}", n, p, W, C)


def test_asymmetric_requests_alone_equal_the_mix_and_a_direct_solve():
    """Requests with an asymmetric C (unfolded tensor-core operand, transposed
    copy of C) served beside symmetric ones: each result equals the request
    served alone and a direct solve on a handle, and its fp64 cost is the
    oracle's objective of the returned allocation."""
    reqs = [(_asym(7300, 120, 6), 8, 31), (synth.clustered(seed=7301, n=150, p=8), 7, 32),
            (_asym(7302, 75, 4), 10, 33), (synth.clustered(seed=7303, n=90, p=5), 9, 34)]
    alone = []
    for inst, gens, seed in reqs:
        with Server(4 * GB, max_active=4, path=PATH_SPLIT_BF16) as s:
            t = s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=gens, seed=seed)
            alone.append(_drain(s, [t])[t])
    with Server(4 * GB, max_active=4, path=PATH_SPLIT_BF16) as s:
        tickets = []
        for k, (inst, gens, seed) in enumerate(reqs):
            tickets.append(s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=gens, seed=seed))
            if k % 2:
                s.step()
        mixed = _drain(s, list(tickets))
    for (inst, gens, seed), a, t in zip(reqs, alone, tickets):
        m = mixed[t]
        np.testing.assert_array_equal(a["hubs"], m["hubs"])
        np.testing.assert_array_equal(a["S"], m["S"])
        assert a["cost_fp32"] == m["cost_fp32"] and a["cost_fp64"] == m["cost_fp64"]
        ref = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, m["S"])
        assert m["cost_fp64"] == pytest.approx(ref, rel=1e-12)
    inst, gens, seed = reqs[0]
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=2, island_size=16, n1=10, path=PATH_SPLIT_BF16)
        direct = gi.solve(gens, seed)
    np.testing.assert_array_equal(direct["hubs"], mixed[tickets[0]]["hubs"])
    assert direct["cost_fp32"] == mixed[tickets[0]]["cost_fp32"]

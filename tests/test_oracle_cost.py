"""Pins of the FP64 oracle's objective, flows, middle nodes and allocation.

Each check ties the oracle to something other than itself: the hand-worked
4-node example, closed forms (p = 1, p = n), the paper's MIP (eq. 1-5) solved
by an independent LP/MIP solver, brute force, and the regrouped three-term
form that the GPU evaluates.
"""
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from oracle import brute, cost
from paper_1704_06258_gb300 import synth


def _hand4(golden_dir):
    rows = [ln.split() for ln in open(os.path.join(golden_dir, "hand4.txt"))
            if ln.strip() and not ln.startswith("#")]
    x = np.array([float(v) for v in next(r for r in rows if r[0] == "x")[1:]])
    W = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "W"], dtype=np.float32)
    chi, alpha, delta = (float(v) for v in next(r for r in rows if r[0] == "params")[1:])
    C = np.abs(x[:, None] - x[None, :]).astype(np.float32)
    return rows, W, C, chi, alpha, delta


def _ints(s):
    return np.array([int(v) for v in s.split(",")])


def test_hand4_costs_terms_flows(golden_dir):
    rows, W, C, chi, alpha, delta = _hand4(golden_dir)
    O, D = cost.flows(W)
    for r in rows:
        if r[0] == "O":
            np.testing.assert_array_equal(O, [float(v) for v in r[1:]])
        elif r[0] == "D":
            np.testing.assert_array_equal(D, [float(v) for v in r[1:]])
        elif r[0] == "cost":
            hubs, h, val = _ints(r[1]), _ints(r[2]), float(r[3])
            cost.check_allocation(4, hubs, h)
            assert cost.pair_cost(W, C, chi, alpha, delta, h) == pytest.approx(val, rel=1e-15)
            assert cost.three_term_cost(W, C, chi, alpha, delta, hubs, h)[0] == pytest.approx(val, rel=1e-15)
        elif r[0] == "terms":
            hubs = _ints(r[1])
            h = cost.nearest_allocation(C, hubs)
            _, tc, td, tt = cost.three_term_cost(W, C, chi, alpha, delta, hubs, h)
            assert (tc, td, tt) == (float(r[2]), float(r[3]), float(r[4]))
        elif r[0] == "scaled":
            h, mode, val = _ints(r[2]), r[3], float(r[4])
            raw = cost.pair_cost(W, C, chi, alpha, delta, h)
            assert cost.scaled_cost(raw, W, mode) == pytest.approx(val, rel=1e-15)
            assert cost.scaled_cost(raw, W, "raw") == raw
        elif r[0] == "middle":
            np.testing.assert_array_equal(cost.middle_nodes(C, int(r[1])), _ints(r[2]))


def test_hand4_brute_force(golden_dir):
    rows, W, C, chi, alpha, delta = _hand4(golden_dir)
    opt = next(r for r in rows if r[0] == "optimum")
    near = next(r for r in rows if r[0] == "nearest_optimum")
    res = brute.brute_force(W, C, chi, alpha, delta, int(opt[1]))
    assert res["opt"][0] == pytest.approx(float(opt[2]), rel=1e-15)
    np.testing.assert_array_equal(res["opt"][1], _ints(opt[3]))
    np.testing.assert_array_equal(res["opt"][2], _ints(opt[4]))
    assert res["nearest"][0] == pytest.approx(float(near[2]), rel=1e-15)
    np.testing.assert_array_equal(res["nearest"][1], _ints(near[3]))


def _mip_optimum(W, C, chi, alpha, delta, p, hub_arcs_only=False):
    """Optimum of the MIP (1)-(5) of §3 (Ernst-Krishnamoorthy form), by HiGHS.

    Variables Z[i,k] (binary) then Y[i,k,l] >= 0 (flow from origin i on hub arc k->l).
    Eq. (1) as printed charges C[i,k] (chi O_i + delta D_i); the instances used
    here have symmetric C, where that equals the oracle's delta D_j C[h(j), j].
    With hub_arcs_only, Y[i,k,l] <= O_i Z[k,k] and Y[i,k,l] <= O_i Z[l,l] keep
    the flow on arcs between open hubs (§3 defines Y as flow between hubs);
    without it constraints (4) also let flow pass through non-hub nodes.
    """
    W = np.asarray(W, np.float64)
    C = np.asarray(C, np.float64)
    n = W.shape[0]
    O, D = W.sum(1), W.sum(0)
    nz, ny = n * n, n * n * n
    zi = lambda i, k: i * n + k
    yi = lambda i, k, l: nz + (i * n + k) * n + l
    c = np.zeros(nz + ny)
    for i in range(n):
        for k in range(n):
            c[zi(i, k)] = C[i, k] * (chi * O[i] + delta * D[i])
            for l in range(n):
                c[yi(i, k, l)] = alpha * C[k, l]
    A = sp.lil_matrix((n + n * n + n * n + 1, nz + ny))
    lb, ub = [], []
    row = 0
    for i in range(n):                      # (2)
        for k in range(n):
            A[row, zi(i, k)] = 1
        lb.append(1); ub.append(1); row += 1
    for i in range(n):                      # (3)
        for k in range(n):
            A[row, zi(i, k)] += 1
            A[row, zi(k, k)] -= 1
            lb.append(-np.inf); ub.append(0); row += 1
    for i in range(n):                      # (4)
        for k in range(n):
            for l in range(n):
                A[row, yi(i, k, l)] += 1
                A[row, yi(i, l, k)] -= 1
            A[row, zi(i, k)] -= O[i]
            for j in range(n):
                A[row, zi(j, k)] += W[i, j]
            lb.append(0); ub.append(0); row += 1
    for k in range(n):                      # (5)
        A[row, zi(k, k)] = 1
    lb.append(p); ub.append(p)
    if hub_arcs_only:
        extra = sp.lil_matrix((2 * ny, nz + ny))
        r = 0
        for i in range(n):
            for k in range(n):
                for l in range(n):
                    for end in (k, l):
                        extra[r, yi(i, k, l)] = 1
                        extra[r, zi(end, end)] = -O[i]
                        r += 1
        A = sp.vstack([A.tocsr(), extra.tocsr()]).tolil()
        lb += [-np.inf] * (2 * ny)
        ub += [0.0] * (2 * ny)
    integrality = np.concatenate([np.ones(nz), np.zeros(ny)])
    bounds = so.Bounds(np.zeros(nz + ny), np.concatenate([np.ones(nz), np.full(ny, np.inf)]))
    res = so.milp(c, integrality=integrality, bounds=bounds,
                  constraints=so.LinearConstraint(A.tocsr(), lb, ub),
                  options={"mip_rel_gap": 1e-12})
    assert res.success, res.message
    return res.fun


def test_hand4_matches_paper_mip(golden_dir):
    rows, W, C, chi, alpha, delta = _hand4(golden_dir)
    for p in (1, 2, 3, 4):
        bf = brute.brute_force(W, C, chi, alpha, delta, p)["opt"][0]
        assert _mip_optimum(W, C, chi, alpha, delta, p) == pytest.approx(bf, rel=1e-9)


@pytest.mark.parametrize("seed,n,p", [(11, 6, 2), (12, 7, 3)])
def test_brute_force_matches_paper_mip_random(seed, n, p):
    inst = synth.tiny(seed=seed, n=n, p=p)
    bf = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, p)
    mip = _mip_optimum(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, p)
    assert mip == pytest.approx(bf["opt"][0], rel=1e-9)
    assert bf["nearest"][0] >= bf["opt"][0]


@pytest.mark.parametrize("seed", [21, 22])
def test_closed_forms_single_hub_and_all_hubs(seed):
    inst = synth.urand200(seed=seed, n=40, p=1)
    W = inst.W.astype(np.float64)
    C = inst.C.astype(np.float64)
    n = inst.n
    O, D = W.sum(1), W.sum(0)
    for k in (0, 7, n - 1):
        h = np.full(n, k)
        expect = inst.chi * (O * C[:, k]).sum() + inst.delta * (D * C[k, :]).sum()
        assert cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, h) == pytest.approx(expect, rel=1e-12)
    h = np.arange(n)
    expect = inst.alpha * (W * C).sum()
    assert cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, h) == pytest.approx(expect, rel=1e-12)


def test_three_term_equals_pair_form_random_allocations():
    inst = synth.urand200(seed=31, n=60, p=7)
    hubs, S = synth.random_population(32, inst.n, inst.p, 8)
    for b in range(8):
        cost.check_allocation(inst.n, hubs[b], S[b])
        a = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, S[b])
        t = cost.three_term_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, np.sort(hubs[b]), S[b])
        assert t[0] == pytest.approx(a, rel=1e-12)


def test_nearest_allocation_is_the_argmin_and_brute_force_nearest():
    inst = synth.tiny(seed=41, n=9, p=3)
    res = brute.brute_force(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, inst.p)
    near_hubs = res["nearest"][1]
    h = cost.nearest_allocation(inst.C, near_hubs)
    for i in range(inst.n):
        d = inst.C[i, near_hubs]
        assert inst.C[i, h[i]] == d.min()
    # For a fixed hub set the nearest allocation can be beaten only by changing
    # the allocation; brute force over allocations is never worse.
    assert res["opt"][0] <= res["nearest"][0]


def test_nearest_allocation_ties_go_to_lowest_node_and_hubs_serve_themselves():
    # Two hubs at the same point: every node ties between them.
    x = np.array([0.0, 3.0, 3.0, 7.0])
    C = np.abs(x[:, None] - x[None, :]).astype(np.float32)
    h = cost.nearest_allocation(C, [2, 1])
    np.testing.assert_array_equal(h, [1, 1, 2, 1])


def test_fig1_encoding(golden_dir):
    rows = {ln.split()[0]: ln.split()[1:] for ln in open(os.path.join(golden_dir, "fig1_encoding.txt"))
            if ln.strip() and not ln.startswith("#")}
    n = int(rows["n"][0])
    H = np.array([int(v) for v in rows["H"]], dtype=bool)
    S = np.array([int(v) for v in rows["S"]]) - 1
    hubs = np.flatnonzero(H)
    cost.check_allocation(n, hubs, S)
    np.testing.assert_array_equal(cost.slots_of(hubs, S), [0, 0, 1, 1, 1, 0, 1])
    with pytest.raises(ValueError):
        bad = S.copy(); bad[1] = 4     # hub 2 (index 1) not serving itself
        cost.check_allocation(n, hubs, bad)
    with pytest.raises(ValueError):
        bad = S.copy(); bad[0] = 0     # node allocated to a spoke
        cost.check_allocation(n, hubs, bad)


def _hand4_nonmetric(golden_dir):
    rows = [ln.split() for ln in open(os.path.join(golden_dir, "hand4_nonmetric.txt"))
            if ln.strip() and not ln.startswith("#")]
    x = np.array([float(v) for v in next(r for r in rows if r[0] == "x")[1:]])
    W = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "W"], dtype=np.float32)
    chi, alpha, delta = (float(v) for v in next(r for r in rows if r[0] == "params")[1:])
    C = np.abs(x[:, None] - x[None, :])
    for r in rows:
        if r[0] == "override":
            a, b, v = int(r[1]), int(r[2]), float(r[3])
            C[a, b] = C[b, a] = v
    return rows, W, C.astype(np.float32), chi, alpha, delta


def test_hand4_nonmetric_costs_by_routing(golden_dir):
    rows, W, C, chi, alpha, delta = _hand4_nonmetric(golden_dir)
    seen = set()
    for r in rows:
        if r[0] != "cost":
            continue
        routing, hubs, h, val = r[1], _ints(r[2]), _ints(r[3]), float(r[4])
        cost.check_allocation(4, hubs, h)
        assert cost.pair_cost(W, C, chi, alpha, delta, h, routing) == pytest.approx(val, rel=1e-15)
        assert cost.three_term_cost(W, C, chi, alpha, delta, hubs, h, routing)[0] == pytest.approx(val, rel=1e-15)
        seen.add(routing)
    assert seen == {"direct", "hubs", "all"}


def _enumerated_paths(A):
    """Cheapest path cost between every ordered pair by trying every sequence
    of distinct intermediate vertices (exponential; tiny sizes only)."""
    import itertools
    m = A.shape[0]
    best = np.full((m, m), np.inf)
    for a in range(m):
        best[a, a] = 0.0
        for b in range(m):
            if a == b:
                continue
            rest = [v for v in range(m) if v not in (a, b)]
            for r in range(len(rest) + 1):
                for mid in itertools.permutations(rest, r):
                    path = (a,) + mid + (b,)
                    best[a, b] = min(best[a, b], sum(A[u, v] for u, v in zip(path, path[1:])))
    return best


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_floyd_warshall_equals_path_enumeration(seed):
    rng = np.random.default_rng(seed)
    A = rng.lognormal(0.0, 1.2, size=(6, 6))
    np.testing.assert_allclose(cost.floyd_warshall(A), _enumerated_paths(A), rtol=1e-14)
    assert (cost.floyd_warshall(A) <= np.where(np.eye(6, dtype=bool), 0.0, A) + 1e-12).all()


def _nonmetric_cases(golden_dir):
    _, W, C, chi, alpha, delta = _hand4_nonmetric(golden_dir)
    cases = [(W, C, chi, alpha, delta, p) for p in (1, 2, 3)]
    for seed, n, p in ((31, 6, 2), (32, 7, 3)):
        inst = synth.latency_like(seed=seed, n=n, p=p, spread=1.0)
        cases.append((inst.W, inst.C, inst.chi, inst.alpha, inst.delta, p))
    return cases


def test_hub_routing_matches_mip_restricted_to_hub_arcs(golden_dir):
    for W, C, chi, alpha, delta, p in _nonmetric_cases(golden_dir):
        bf = brute.brute_force(W, C, chi, alpha, delta, p, routing="hubs")
        mip = _mip_optimum(W, C, chi, alpha, delta, p, hub_arcs_only=True)
        assert mip == pytest.approx(bf["opt"][0], rel=1e-9)
        assert bf["opt"][0] <= brute.brute_force(W, C, chi, alpha, delta, p)["opt"][0]


def test_all_node_routing_matches_mip_as_printed(golden_dir):
    for W, C, chi, alpha, delta, p in _nonmetric_cases(golden_dir):
        bf = brute.brute_force(W, C, chi, alpha, delta, p, routing="all")
        assert _mip_optimum(W, C, chi, alpha, delta, p) == pytest.approx(bf["opt"][0], rel=1e-9)


def test_routing_changes_nothing_on_euclidean_instances():
    inst = synth.urand200(seed=41, n=60, p=6)
    hubs, S = synth.random_population(42, inst.n, inst.p, 5)
    for s in S:
        direct = cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s)
        for routing in ("hubs", "all"):
            assert cost.pair_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, s, routing) == \
                pytest.approx(direct, rel=1e-6)
    tiny = synth.tiny(seed=43, n=7, p=3)
    opts = [brute.brute_force(tiny.W, tiny.C, tiny.chi, tiny.alpha, tiny.delta, 3, r)["opt"][0]
            for r in ("direct", "hubs", "all")]
    assert opts[1] == pytest.approx(opts[0], rel=1e-6) and opts[2] == pytest.approx(opts[0], rel=1e-6)

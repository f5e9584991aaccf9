"""FP64 objective, flows, initial solution and allocation (oracle; test use only).

Definitions follow the paper:

* Objective, §3 eq. (1): for a single allocation h (h[k] = k for each hub k)
  the cost of routing W[i, j] from i to j is collection at rate chi on arc
  (i, h(i)), transfer at discount alpha on the hub arc (h(i), h(j)) and
  distribution at rate delta on (h(j), j) -- the path cost written out in
  §6.2.  Eq. (4) lets hub-to-hub flow take any path; with C satisfying the
  triangle inequality (every Euclidean instance) the direct hub arc is a
  shortest path, which is `routing="direct"`.  For C without it (§6.1's
  PlanetLab latencies) the transfer leg takes a shortest path:
  `routing="hubs"` over arcs between open hubs only (§3 defines Y^i_kl as
  flow between hubs k and l), `routing="all"` over arcs between any nodes (what
  constraints (4) alone admit: a non-hub node is a zero-balance transshipment
  node there).  Both give a same-hub pair a zero transfer leg (flow from k to
  k needs no Y in eq. 4).
* O_i and D_j are the originating and destined flows of §3 (row and column
  sums of W).
* Middle nodes, §4.1: the p nodes with the smallest d_i = sum_j C[i, j]
  (ties broken towards the lower node id); then every node goes to its
  nearest hub.
* Nearest allocation, §4.1 and §5: h(i) = argmin over open hubs k of C[i, k];
  ties go to the lowest node id and every hub serves itself (eq. 2-3).

Pins (tests/test_oracle_*.py): hand-worked 4-node values
(tests/golden/hand4.txt); closed forms for p = 1 and p = n; brute force over
all hub sets and all allocations; the optimum of the paper's MIP, eq. (1)-(5),
solved by an LP/MIP solver on tiny instances; the three-term form (with the
dense product M = W A) against the pair form.
"""
from __future__ import annotations

import math

import numpy as np


def _f64(x):
    return np.asarray(x, dtype=np.float64)


def flows(W):
    """(O, D) in FP64: O_i = sum_j W[i, j], D_j = sum_i W[i, j] (§3)."""
    W = _f64(W)
    n = W.shape[0]
    O = np.array([math.fsum(W[i, :]) for i in range(n)])
    D = np.array([math.fsum(W[:, j]) for j in range(n)])
    return O, D


def check_allocation(n, hubs, h):
    """Raise ValueError unless (hubs, h) is a valid single allocation (eq. 2, 3, 5)."""
    hubs = np.asarray(hubs)
    h = np.asarray(h)
    if len(set(hubs.tolist())) != len(hubs):
        raise ValueError("hubs not distinct")
    if hubs.min() < 0 or hubs.max() >= n:
        raise ValueError("hub out of range")
    hs = set(hubs.tolist())
    for i in range(n):
        if int(h[i]) not in hs:
            raise ValueError(f"node {i} allocated to non-hub {h[i]}")
    for k in hubs:
        if h[k] != k:
            raise ValueError(f"hub {k} not allocated to itself")


def floyd_warshall(A):
    """Shortest-path costs over a complete digraph with arc costs A (FP64).

    The textbook recurrence: after step k, D[a, b] is the cheapest path from a
    to b whose intermediate vertices are among the first k + 1; D[a, a] = 0.
    """
    D = _f64(A).copy()
    np.fill_diagonal(D, 0.0)
    for k in range(D.shape[0]):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def transfer_costs(C, h, routing="direct"):
    """n x n matrix T with T[a, b] the unit cost of the transfer leg from hub a
    to hub b (entries between non-hubs are unused).

    direct: C itself; hubs: shortest paths over arcs between the open hubs
    (the distinct values of h); all: shortest paths over arcs between any
    nodes.
    """
    C = _f64(C)
    if routing == "direct":
        return C
    if routing == "all":
        return floyd_warshall(C)
    if routing != "hubs":
        raise ValueError(routing)
    hubs = np.unique(np.asarray(h, dtype=np.int64))
    T = C.copy()
    T[np.ix_(hubs, hubs)] = floyd_warshall(C[np.ix_(hubs, hubs)])
    return T


def pair_cost(W, C, chi, alpha, delta, h, routing="direct"):
    """Objective (1) summed pair by pair in FP64.

    cost = sum_i sum_j W[i,j] * (chi*C[i,h(i)] + alpha*T[h(i),h(j)] + delta*C[h(j),j])
    with T the transfer-leg costs of `routing` (T = C for the direct arc).
    """
    W = _f64(W)
    C = _f64(C)
    h = np.asarray(h, dtype=np.int64)
    n = W.shape[0]
    idx = np.arange(n)
    T = transfer_costs(C, h, routing)
    collect = C[idx, h]                  # C[i, h(i)]
    transfer = T[h[:, None], h[None, :]]  # T[h(i), h(j)]
    distribute = C[h, idx]               # C[h(j), j]
    per_pair = W * (chi * collect[:, None] + alpha * transfer + delta * distribute[None, :])
    return math.fsum(np.sum(per_pair, axis=1))


def scaled_cost(value, W, scale="raw"):
    """The fitness as the benchmarks of §4.3 report it: "raw" (PlanetLab),
    "milli" (the cost times 10^-3, AP and Urand) or "per_flow" (the cost
    divided by the total flow sum_ij W[i,j], CAB)."""
    if scale == "raw":
        return float(value)
    if scale == "milli":
        return float(value) * 1e-3
    if scale == "per_flow":
        return float(value) / math.fsum(_f64(W).ravel())
    raise ValueError(scale)


def three_term_cost(W, C, chi, alpha, delta, hubs, h, routing="direct"):
    """The same objective regrouped as the GPU evaluates it.

    chi * sum_i O_i C[i,h(i)] + delta * sum_j D_j C[h(j),j]
      + alpha * sum_i sum_l M[i,l] T[h(i), hubs[l]],   M = W A,
    with A the n x p one-hot matrix A[j, l] = [h(j) == hubs[l]] and T the
    transfer-leg costs of `routing`.
    Returns (total, collect_term, distribute_term, transfer_term).
    """
    W = _f64(W)
    C = _f64(C)
    hubs = np.asarray(hubs, dtype=np.int64)
    h = np.asarray(h, dtype=np.int64)
    n = W.shape[0]
    p = len(hubs)
    O, D = flows(W)
    idx = np.arange(n)
    t_collect = chi * math.fsum(O * C[idx, h])
    t_distribute = delta * math.fsum(D * C[h, idx])
    A = np.zeros((n, p))
    for l in range(p):
        A[h == hubs[l], l] = 1.0
    M = W @ A
    T = transfer_costs(C, hubs, routing)
    t_transfer = alpha * math.fsum(np.sum(M * T[h[:, None], hubs[None, :]], axis=1))
    return t_collect + t_distribute + t_transfer, t_collect, t_distribute, t_transfer


def middle_nodes(C, p):
    """§4.1: the p nodes with the smallest d_i = sum_j C[i,j], ascending node ids."""
    C = _f64(C)
    d = np.array([math.fsum(C[i, :]) for i in range(C.shape[0])])
    order = sorted(range(len(d)), key=lambda i: (d[i], i))
    return np.array(sorted(order[:p]), dtype=np.int64)


def nearest_allocation(C, hubs):
    """h(i) = the open hub k minimising C[i,k]; lowest node id on ties; hubs serve themselves.

    The comparison is done on the instance's own FP32 values (C is FP32), so
    the decision is the one any exact comparison of those values makes.
    """
    C = np.asarray(C)
    hubs = np.sort(np.asarray(hubs, dtype=np.int64))
    n = C.shape[0]
    h = np.empty(n, dtype=np.int64)
    for i in range(n):
        best = hubs[0]
        for k in hubs[1:]:
            if C[i, k] < C[i, best]:
                best = k
        h[i] = best
    h[hubs] = hubs
    return h


def slots_of(hubs_sorted, h):
    """Rank of h(i) within the ascending hub list (the library's u8 slot code)."""
    pos = {int(k): r for r, k in enumerate(hubs_sorted)}
    return np.array([pos[int(x)] for x in h], dtype=np.int64)


def initial_solution(C, p):
    """Middle-node hubs plus nearest allocation (§4.1)."""
    hubs = middle_nodes(C, p)
    return hubs, nearest_allocation(C, hubs)

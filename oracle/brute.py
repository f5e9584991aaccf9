"""Exhaustive search over hub sets and allocations (oracle; test use only).

For tiny n this enumerates every set of p hubs and every single allocation
of the spokes to those hubs, evaluating objective (1) of §3 with the transfer
leg of `routing` (cost.transfer_costs: the direct hub arc, or shortest paths
over hub arcs or over all arcs), and returns both the global optimum and the
best solution whose allocation is the nearest-hub one (§4.1).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import cost as _cost


def _batch_costs(W, C, T, chi, alpha, delta, H):
    """Pair-form objective for every allocation row of H ([A, n] node ids), FP64;
    T holds the transfer-leg costs between hubs."""
    n = W.shape[0]
    idx = np.arange(n)
    collect = C[idx[None, :], H]                     # [A, n]  C[i, h(i)]
    transfer = T[H[:, :, None], H[:, None, :]]       # [A, n, n]
    distribute = C[H, idx[None, :]]                  # [A, n]  C[h(j), j]
    per = W[None] * (chi * collect[:, :, None] + alpha * transfer + delta * distribute[:, None, :])
    return per.reshape(per.shape[0], -1).sum(axis=1)


def brute_force(W, C, chi, alpha, delta, p, routing="direct"):
    """Returns dict(opt=(cost, hubs, h), nearest=(cost, hubs, h))."""
    W = np.asarray(W, dtype=np.float64)
    Cf = np.asarray(C, dtype=np.float64)
    n = W.shape[0]
    best = (np.inf, None, None)
    best_near = (np.inf, None, None)
    for hubs in itertools.combinations(range(n), p):
        hubs = np.array(hubs)
        spokes = np.array([i for i in range(n) if i not in set(hubs.tolist())], dtype=np.int64)
        allocs = np.array(list(itertools.product(hubs.tolist(), repeat=len(spokes))), dtype=np.int64)
        H = np.empty((len(allocs), n), dtype=np.int64)
        H[:, hubs] = hubs
        if len(spokes):
            H[:, spokes] = allocs
        T = _cost.transfer_costs(Cf, hubs, routing)
        costs = _batch_costs(W, Cf, T, chi, alpha, delta, H)
        a = int(np.argmin(costs))
        if costs[a] < best[0]:
            best = (float(costs[a]), hubs, H[a].copy())
        hn = _cost.nearest_allocation(C, hubs)
        cn = _cost.pair_cost(W, Cf, chi, alpha, delta, hn, routing)
        if cn < best_near[0]:
            best_near = (cn, hubs, hn)
    return {"opt": best, "nearest": best_near}

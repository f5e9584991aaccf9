"""The island GA of §4-§5, step by step, on boolean hub masks (oracle; test use only).

The paper names the operators but leaves their details open; the readings
used here (and by the library) are:

* A chromosome is the pair (H, S) of §4.1.  Only H (the hub mask) is evolved;
  S is recomputed by nearest allocation after every change (§5: each thread
  checks that every node is assigned to its nearest hub).
* Hub <-> spoke exchange (the move that builds the initial population from
  the ancestor, §4.1, and -- read the same way -- the mutation of §4.2, whose
  literal "permutation of two hubs" would not change H): with h open nodes,
  i = below(h) and j = below(n - h) are drawn; when 0 < h < n the i-th open
  node is closed and the j-th closed node is opened, both counted in
  ascending node order on the mask before the change.  Both words are drawn
  whatever h is.
* Single-point crossover (§4.2, §5): the pair (2m, 2m+1) of an island draws
  one cut c = 1 + below(n - 1); each child keeps the bits [0, c) of one parent
  and takes [c, n) from the other.
* Correction (§4.2): while more than p nodes are open, close the
  below(h)-th open node; while fewer, open the below(n - h)-th closed node.
* Selection (§5): island r's ancestor becomes its child with the smallest
  fitness (lowest member index on ties; a NaN fitness, which has no order,
  ranks after every number).  The best-ever solution is replaced
  only by a strictly smaller fitness, islands scanned in ascending order.
  Every N1 generations (the outer loop) every island's ancestor becomes the
  ancestor of the island whose ancestor fitness is smallest (lowest island on
  ties).
* Random numbers come from Philox4x32-10 draw streams keyed by the seed and
  addressed by (generation, chromosome, operator) -- see oracle.philox.

Pins (tests/test_oracle_ga.py): validity invariants (popcount p, hub
self-allocation, argmin allocation), exhaustive checks of each operator on
tiny masks (every cut, every exchange), the uniformity of the draws, and the
full GA reaching the brute-force best nearest-allocation optimum on the
10-node instance.
"""
from __future__ import annotations

import numpy as np

from . import cost as _cost
from .philox import (DrawStream, OP_CORRECTION, OP_CROSSOVER, OP_MUTATION,
                     OP_PERTURB)


def kth_open(mask, k):
    return int(np.flatnonzero(mask)[k])


def kth_closed(mask, k):
    return int(np.flatnonzero(~mask)[k])


def exchange(mask, stream):
    """One hub <-> spoke exchange, in place."""
    n = mask.size
    h = int(mask.sum())
    i = stream.below(h)
    j = stream.below(n - h)
    if 0 < h < n:
        a = kth_open(mask, i)
        b = kth_closed(mask, j)
        mask[a] = False
        mask[b] = True
    return mask


def crossover(pa, pb, stream):
    """Children of the pair (pa, pb) with one random cut."""
    n = pa.size
    c = 1 + stream.below(n - 1)
    ca = np.concatenate([pa[:c], pb[c:]])
    cb = np.concatenate([pb[:c], pa[c:]])
    return ca, cb, c


def correct(mask, p, stream):
    """Bring the number of open nodes back to p, in place."""
    n = mask.size
    h = int(mask.sum())
    while h > p:
        mask[kth_open(mask, stream.below(h))] = False
        h -= 1
    while h < p:
        mask[kth_closed(mask, stream.below(n - h))] = True
        h += 1
    return mask


def make_children(ancestors, seed, g, p, P, island_offset=0):
    """One generation of offspring: exchange -> crossover -> mutation -> correction.

    ancestors: bool [R, n].  Returns bool [R*P, n]; chromosome q = r*P + j
    belongs to island r.  The draw streams are addressed by the global index
    (island_offset*P + q), so a slice of the islands draws what the whole
    population draws for them.
    """
    R, n = ancestors.shape
    B = R * P
    q0 = island_offset * P
    parents = np.empty((B, n), dtype=bool)
    for q in range(B):
        parents[q] = exchange(ancestors[q // P].copy(), DrawStream(seed, g, q0 + q, OP_PERTURB))
    children = parents.copy()
    for q in range(0, B, 2):
        ca, cb, _ = crossover(parents[q], parents[q + 1], DrawStream(seed, g, q0 + q, OP_CROSSOVER))
        children[q], children[q + 1] = ca, cb
    for q in range(B):
        exchange(children[q], DrawStream(seed, g, q0 + q, OP_MUTATION))
        correct(children[q], p, DrawStream(seed, g, q0 + q, OP_CORRECTION))
    return children


def allocate_all(C, masks):
    """(hubs [B,p] ascending, h [B,n] node ids, slot [B,n]) by nearest allocation."""
    B, n = masks.shape
    hubs = np.stack([np.flatnonzero(m) for m in masks])
    h = np.stack([_cost.nearest_allocation(C, hb) for hb in hubs])
    slot = np.stack([_cost.slots_of(hb, hh) for hb, hh in zip(hubs, h)])
    return hubs, h, slot


class State:
    """Island GA state: ancestors, their fitness, best-ever."""

    def __init__(self, ancestors, anc_fit, best, best_fit):
        self.ancestors = ancestors.copy()
        self.anc_fit = np.asarray(anc_fit, dtype=np.float64).copy()
        self.best = best.copy()
        self.best_fit = float(best_fit)


def _rank(x):
    """Selection key: NaN ranks after every number."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.isnan(x), np.inf, x)


def select(state, children, fitness, g, P, N1, elitist=False):
    """Inner-loop selection and the outer-loop merge of §5, in place on `state`
    (N1 = 0: no merge; a population split over several GPUs merges across
    them instead, see merge_shards)."""
    R = state.ancestors.shape[0]
    fitness = _rank(fitness)
    for r in range(R):
        f = fitness[r * P:(r + 1) * P]
        j = int(np.argmin(f))           # first minimum: lowest member index
        if elitist and not (f[j] < state.anc_fit[r]):
            continue
        state.ancestors[r] = children[r * P + j]
        state.anc_fit[r] = f[j]
    rb = int(np.argmin(_rank(state.anc_fit)))  # first minimum: lowest island
    if state.anc_fit[rb] < state.best_fit:
        state.best = state.ancestors[rb].copy()
        state.best_fit = float(state.anc_fit[rb])
    if N1 > 0 and (g + 1) % N1 == 0:
        state.ancestors[:] = state.ancestors[rb]
        state.anc_fit[:] = state.anc_fit[rb]
    return state


def merge_shards(states, island_counts):
    """The §5 merge across shards of one island population: every island of
    every shard takes the ancestor of the island with the smallest ancestor
    fitness over all shards (NaN last; lowest global island index on ties).
    `states` are the shards' States in global island order."""
    best = None
    base = 0
    for st, R in zip(states, island_counts):
        f = _rank(st.anc_fit)
        r = int(np.argmin(f))
        if best is None or f[r] < best[0]:
            best = (f[r], st.ancestors[r].copy(), float(st.anc_fit[r]))
        base += R
    for st in states:
        st.ancestors[:] = best[1]
        st.anc_fit[:] = best[2]
    return best[1], best[2]


def solve(inst, generations, seed, R=1, P=64, N1=10, elitist=False, fitness_fn=None, routing="direct"):
    """The whole GA on one instance with FP64 fitness; returns (hubs, h, cost, state).

    `routing` is the transfer leg of the objective (cost.transfer_costs)."""
    W, C = inst.W, inst.C
    n, p = inst.n, inst.p
    if fitness_fn is None:
        def fitness_fn(h):
            return _cost.pair_cost(W, C, inst.chi, inst.alpha, inst.delta, h, routing)
    hubs0, h0 = _cost.initial_solution(C, p)
    mask0 = np.zeros(n, dtype=bool)
    mask0[hubs0] = True
    f0 = fitness_fn(h0)
    state = State(np.tile(mask0, (R, 1)), np.full(R, f0), mask0, f0)
    for g in range(generations):
        children = make_children(state.ancestors, seed, g, p, P)
        _, h, _ = allocate_all(C, children)
        fit = np.array([fitness_fn(hh) for hh in h])
        select(state, children, fit, g, P, N1, elitist)
    hubs = np.flatnonzero(state.best)
    h = _cost.nearest_allocation(C, hubs)
    return hubs, h, _cost.pair_cost(W, C, inst.chi, inst.alpha, inst.delta, h, routing), state

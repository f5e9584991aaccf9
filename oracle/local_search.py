"""Allocation local search (oracle; test use only).

The GA allocates every spoke to its nearest open hub (§4.1, §5), which is
not always the cheapest allocation for a fixed hub set: a spoke that sends
much of its flow through a farther hub can be cheaper there.  This search
improves an allocation for fixed hubs by single reallocations:

* a sweep visits the spokes in ascending node order (hubs keep serving
  themselves, eq. 3);
* for spoke i it computes, for every other open hub b (ascending node id),
  the change of objective (1) when i moves from h(i) to b -- here literally
  cost(h with h(i) = b) - cost(h), each cost summed pair by pair in FP64;
* it moves i to the hub with the most negative change (the lowest node id
  among equal changes), if that change is negative, before visiting the
  next spoke;
* sweeps repeat until one moves nothing or `max_sweeps` have run.

The result is a local optimum for single reallocations whenever the search
stops on a sweep without moves.  Pins (tests/test_oracle_local_search.py):
exhaustive single-move checks of that property, the brute-force optimum
being a fixed point, monotone cost, and a hand-worked move.
"""
from __future__ import annotations

import numpy as np

from . import cost as _cost


def local_search(W, C, chi, alpha, delta, hubs, h, max_sweeps, routing="direct"):
    """Returns (h, sweeps run, moves made); h is not modified."""
    h = np.array(h, dtype=np.int64)
    hubs = np.sort(np.asarray(hubs, dtype=np.int64))
    hubset = set(hubs.tolist())
    n = h.size
    moves = 0
    sweeps = 0
    for _ in range(max_sweeps):
        sweeps += 1
        moved = False
        for i in range(n):
            if i in hubset:
                continue
            base = _cost.pair_cost(W, C, chi, alpha, delta, h, routing)
            best_b, best_d = -1, 0.0
            for b in hubs:
                if b == h[i]:
                    continue
                h2 = h.copy()
                h2[i] = b
                d = _cost.pair_cost(W, C, chi, alpha, delta, h2, routing) - base
                if d < best_d:
                    best_b, best_d = int(b), d
            if best_b >= 0:
                h[i] = best_b
                moves += 1
                moved = True
        if not moved:
            break
    return h, sweeps, moves

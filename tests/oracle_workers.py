"""Process-pool workers that run the oracle for the GPU tests (spawned
processes: no CUDA state, only numpy and oracle/).

The instance is handed to every worker once, through the pool initializer."""
import numpy as np

from oracle import cost
from oracle.local_search import local_search

_INST = {}


def init(W, C, chi, alpha, delta):
    _INST.update(W=W, C=C, chi=chi, alpha=alpha, delta=delta)


def run_local_search(args):
    """The oracle's search from one start: (h, sweeps, moves)."""
    hubs, start, max_sweeps, routing = args
    return local_search(_INST["W"], _INST["C"], _INST["chi"], _INST["alpha"], _INST["delta"], hubs, start,
                        max_sweeps, routing)


def single_move_changes(args):
    """Objective change of every single reallocation of spoke i away from its
    hub in allocation h, each as the difference of two pair-form costs:
    [(hub, cost(h with h(i) = hub) - cost(h)), ...] and cost(h)."""
    h, i, hubs = args
    W, C, chi, alpha, delta = _INST["W"], _INST["C"], _INST["chi"], _INST["alpha"], _INST["delta"]
    base = cost.pair_cost(W, C, chi, alpha, delta, h)
    out = []
    for b in hubs:
        if b == h[i]:
            continue
        h2 = np.array(h, copy=True)
        h2[i] = b
        out.append((int(b), cost.pair_cost(W, C, chi, alpha, delta, h2) - base))
    return out, base

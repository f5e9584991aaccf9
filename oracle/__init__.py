"""Plain FP64 CPU oracle for the USApHMP hot path (TEST INFRASTRUCTURE ONLY).

This package restates, slowly and directly, what the GPU library computes:
the single-allocation p-hub median objective (§3, eq. 1), the middle-node
initial solution and nearest-hub allocation (§4.1), the GA operators (§4.2)
and the island GA loop (§5).  It shares no code with the CUDA path.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg (and its
``--impl reference`` arm) may import or run anything in this package.  The
library itself never falls back to it.

Pins (what fixes each function independently of itself) are listed in each
module's header; every function here is pinned, none is "parity unpinned".
"""

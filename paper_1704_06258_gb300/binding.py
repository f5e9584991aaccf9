"""ctypes binding of libusaphmp.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/usaphmp.h; the
arithmetic runs in the library's CUDA kernels.  Device pointers are plain
integers (e.g. ``torch.Tensor.data_ptr()``) and streams are raw
``cudaStream_t`` values (e.g. ``torch.cuda.current_stream().cuda_stream``).
There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libusaphmp.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "usaphmp.h")

PATH_PLAIN_FP32 = 0
PATH_SPLIT_BF16 = 1
PATH_FP64_REF = 2
ROUTE_DIRECT = 0
ROUTE_HUB_PATHS = 1
SCALE_RAW = 0
SCALE_MILLI = 1
SCALE_PER_FLOW = 2

ERRORS = {-1: "EINVAL", -2: "EINVAL_CHROM", -3: "ENOMEM", -4: "ECUDA", -5: "ETIMEOUT", -6: "EBUSY", -7: "EIO",
          -8: "ECANCELED"}

c_i32, c_i64, c_u64, c_f64, c_f32, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_float, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [("islands", c_i32), ("island_size", c_i32), ("n1", c_i32), ("path", c_i32),
                ("elitist", c_i32), ("use_graph", c_i32), ("routing", c_i32), ("scale", c_i32),
                ("local_search", c_i32), ("island_offset", c_i32)]


class Result(ctypes.Structure):
    _fields_ = [("hubs", ctypes.POINTER(c_i32)), ("S", ctypes.POINTER(c_i32)), ("cost_fp64", c_f64),
                ("cost_fp32", c_f32), ("evals", c_i64), ("ms", c_f64)]


class Tile(ctypes.Structure):
    _fields_ = [("ntile", c_i32), ("stages", c_i32), ("raster", c_i32), ("pair", c_i32)]


class Info(ctypes.Structure):
    _fields_ = [("n", c_i32), ("p", c_i32), ("ldw", c_i32), ("ns", c_i32), ("c_symmetric", c_i32),
                ("tc_folded", c_i32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("ticks", c_i64), ("tick_ms_total", c_f64), ("tick_ms_max", c_f64), ("admitted", c_i64),
                ("admit_wait_ms_total", c_f64), ("admit_wait_ms_max", c_f64), ("admit_ms_total", c_f64),
                ("graph_builds", c_i64)]


class UsaphmpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


_SIGS = {
    "usaphmp_create": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_f64, c_f64, c_f64, ctypes.POINTER(c_vp)]),
    "usaphmp_create_dev": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_f64, c_f64, c_f64, c_vp, ctypes.POINTER(c_vp)]),
    "usaphmp_set_params": (c_i32, [c_vp, ctypes.POINTER(Params)]),
    "usaphmp_get_params": (c_i32, [c_vp, ctypes.POINTER(Params)]),
    "usaphmp_eval": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "usaphmp_eval_dev": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_solve": (c_i32, [c_vp, c_i32, c_u64, ctypes.POINTER(Result)]),
    "usaphmp_destroy": (None, [c_vp]),
    "usaphmp_last_error": (ctypes.c_char_p, []),
    "usaphmp_layout": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    "usaphmp_initial_dev": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_children_dev": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_u64, c_i32, c_vp, c_vp, c_vp]),
    "usaphmp_allocate_dev": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "usaphmp_eval_slots_dev": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_select_dev": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_rescore_fp64_dev": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_ga_begin": (c_i32, [c_vp, c_u64, c_vp]),
    "usaphmp_ga_run": (c_i32, [c_vp, c_i32, c_vp]),
    "usaphmp_ga_result": (c_i32, [c_vp, ctypes.POINTER(Result), c_vp]),
    "usaphmp_ga_run_profiled": (c_i32, [c_vp, c_i32, c_vp, ctypes.POINTER(c_f64)]),
    "usaphmp_rescore_fp64_noalloc": (c_i32, [c_i32, c_i32, c_i32, c_vp, c_vp, c_f64, c_f64, c_f64, c_vp, c_vp,
                                             c_vp, c_vp]),
    "usaphmp_server_create": (c_i32, [c_i64, c_i32, c_i32, ctypes.POINTER(c_vp)]),
    "usaphmp_server_submit": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_f64, c_f64, c_f64, c_i32, c_i32, c_i32,
                                      c_u64, ctypes.POINTER(c_i64)]),
    "usaphmp_server_step": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    "usaphmp_server_poll": (c_i32, [c_vp, c_i64, ctypes.POINTER(Result)]),
    "usaphmp_server_footprint": (c_i32, [c_i32, c_i32, c_i32, c_i32, ctypes.POINTER(c_i64)]),
    "usaphmp_server_destroy": (None, [c_vp]),
    "usaphmp_server_cancel": (c_i32, [c_vp, c_i64]),
    "usaphmp_server_stats": (c_i32, [c_vp, ctypes.POINTER(ServerStats)]),
    "usaphmp_debug_fail_allocations": (c_i32, [c_i32]),
    "usaphmp_selftest_wait_timeout": (c_i32, [c_i64, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(c_i64)]),
    "usaphmp_ga_islands": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_ga_population": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "usaphmp_ga_state_bytes": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "usaphmp_ga_save": (c_i32, [c_vp, c_vp, c_i64, c_vp]),
    "usaphmp_ga_load": (c_i32, [c_vp, c_vp, c_i64, c_vp]),
    "usaphmp_ga_merge": (c_i32, [c_vp, c_vp, c_f32, c_vp]),
    "usaphmp_local_search_dev": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "usaphmp_set_tile": (c_i32, [c_vp, ctypes.POINTER(Tile)]),
    "usaphmp_get_tile": (c_i32, [c_vp, ctypes.POINTER(Tile)]),
    "usaphmp_get_info": (c_i32, [c_vp, ctypes.POINTER(Info)]),
    "usaphmp_autotune": (c_i32, [c_vp, c_i32, ctypes.c_char_p, ctypes.POINTER(Tile), ctypes.POINTER(c_f64),
                                 ctypes.POINTER(c_f64), ctypes.POINTER(c_i32)]),
    "usaphmp_tile_cache_lookup": (c_i32, [ctypes.c_char_p, ctypes.c_char_p, c_i32, c_i32, c_i32,
                                          ctypes.POINTER(Tile), ctypes.POINTER(c_f64)]),
    "usaphmp_tile_cache_store": (c_i32, [ctypes.c_char_p, ctypes.c_char_p, c_i32, c_i32, c_i32,
                                         ctypes.POINTER(Tile), c_f64]),
}

STAGES = ("offspring", "allocation", "transfer", "reduce_select", "unused", "generation")

_lib = None


def header_functions(path=HEADER):
    """Names of the functions declared in a public header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(usaphmp_\w+)\s*\(", text)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != 0:
        raise UsaphmpError(rc, (lib().usaphmp_last_error() or b"").decode())


def _ptr(a):
    # the buffer's address as an int (c_void_p arguments accept it; cheaper
    # than building a ctypes pointer object on every call)
    return a.__array_interface__["data"][0]


def debug_fail_allocations(after):
    """usaphmp_debug_fail_allocations (testing hook)."""
    check(lib().usaphmp_debug_fail_allocations(after))


def selftest_wait_timeout(limit_ns):
    """usaphmp_selftest_wait_timeout: (return code, status word, elapsed ns)."""
    st, el = ctypes.c_uint32(), c_i64()
    rc = lib().usaphmp_selftest_wait_timeout(int(limit_ns), ctypes.byref(st), ctypes.byref(el))
    return rc, st.value, el.value


def rescore_fp64_noalloc(n, p, B, W_ptr, C_ptr, chi, alpha, delta, hubs_ptr, slot_ptr, cost_ptr, stream=0):
    """usaphmp_rescore_fp64_noalloc: no handle, no allocation (dense W, C, slot)."""
    check(lib().usaphmp_rescore_fp64_noalloc(n, p, B, W_ptr, C_ptr, chi, alpha, delta, hubs_ptr, slot_ptr,
                                             cost_ptr, stream))


def _tile_dict(t):
    return {"ntile": int(t.ntile), "stages": int(t.stages), "raster": int(t.raster), "pair": int(t.pair)}


def tile_cache_lookup(path, device, n, p, B):
    """usaphmp_tile_cache_lookup: the cached tile dict (with "ms") or None."""
    t, ms = Tile(), c_f64()
    rc = lib().usaphmp_tile_cache_lookup(os.fsencode(path), device.encode(), n, p, B, ctypes.byref(t),
                                         ctypes.byref(ms))
    if rc < 0:
        check(rc)
    if rc == 0:
        return None
    d = _tile_dict(t)
    d["ms"] = ms.value
    return d


def tile_cache_store(path, device, n, p, B, ntile, stages, raster, ms, pair=0):
    """usaphmp_tile_cache_store."""
    t = Tile(ntile, stages, raster, pair)
    check(lib().usaphmp_tile_cache_store(os.fsencode(path), device.encode(), n, p, B, ctypes.byref(t), ms))


class Instance:
    """One USApHMP instance resident on the GPU (a ``usaphmp_t``)."""

    def __init__(self, W, C, p, chi=3.0, alpha=0.75, delta=2.0):
        W = np.ascontiguousarray(W, dtype=np.float32)
        C = np.ascontiguousarray(C, dtype=np.float32)
        if W.ndim != 2 or W.shape[0] != W.shape[1] or C.shape != W.shape:
            raise ValueError("W and C must be n x n")
        self.n, self.p = int(W.shape[0]), int(p)
        self.chi, self.alpha, self.delta = float(chi), float(alpha), float(delta)
        h = c_vp()
        check(lib().usaphmp_create(self.n, self.p, _ptr(W), _ptr(C), self.chi, self.alpha, self.delta,
                                   ctypes.byref(h)))
        self.h = h
        ns, nw = c_i32(), c_i32()
        check(lib().usaphmp_layout(self.h, ctypes.byref(ns), ctypes.byref(nw)))
        self.ns, self.nw = ns.value, nw.value

    @classmethod
    def from_instance(cls, inst):
        return cls(inst.W, inst.C, inst.p, inst.chi, inst.alpha, inst.delta)

    def close(self):
        if getattr(self, "h", None):
            lib().usaphmp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # parameters
    @property
    def params(self):
        prm = Params()
        check(lib().usaphmp_get_params(self.h, ctypes.byref(prm)))
        return {f: getattr(prm, f) for f, _ in Params._fields_}

    def set_params(self, **kw):
        cur = self.params
        cur.update(kw)
        prm = Params(**cur)
        check(lib().usaphmp_set_params(self.h, ctypes.byref(prm)))

    def set_tile(self, ntile, stages, raster, pair=0):
        """usaphmp_set_tile: tile shape of the tensor-core evaluator."""
        t = Tile(ntile, stages, raster, pair)
        check(lib().usaphmp_set_tile(self.h, ctypes.byref(t)))

    def info(self):
        """usaphmp_get_info as a dict."""
        t = Info()
        check(lib().usaphmp_get_info(self.h, ctypes.byref(t)))
        return {name: int(getattr(t, name)) for name, _ in Info._fields_}

    def get_tile(self):
        t = Tile()
        check(lib().usaphmp_get_tile(self.h, ctypes.byref(t)))
        return _tile_dict(t)

    def autotune(self, reps=20, cache=None):
        """usaphmp_autotune: times the tile shapes, keeps the fastest.

        Returns the chosen shape with "ms" (its mean launch time), "default_ms"
        and "from_cache".  Resets the GA state (call ga_begin/solve after)."""
        t, ms, dms, fc = Tile(), c_f64(), c_f64(), c_i32()
        check(lib().usaphmp_autotune(self.h, reps, os.fsencode(cache) if cache else None, ctypes.byref(t),
                                     ctypes.byref(ms), ctypes.byref(dms), ctypes.byref(fc)))
        d = _tile_dict(t)
        d.update(ms=ms.value, default_ms=dms.value, from_cache=bool(fc.value))
        return d

    # public calls
    def eval(self, hubs, S):
        hubs = np.ascontiguousarray(hubs, dtype=np.int32)
        S = np.ascontiguousarray(S, dtype=np.int32)
        B = hubs.shape[0]
        if hubs.shape != (B, self.p) or S.shape != (B, self.n):
            raise ValueError("hubs must be [B, p] and S [B, n]")
        out = np.empty(B, dtype=np.float64)
        check(lib().usaphmp_eval(self.h, B, _ptr(hubs), _ptr(S), _ptr(out)))
        return out

    def eval_dev(self, B, hubs_ptr, S_ptr, fitness_ptr, stream=0):
        check(lib().usaphmp_eval_dev(self.h, B, hubs_ptr, S_ptr, fitness_ptr, stream))

    def solve(self, generations, seed):
        hubs = np.empty(self.p, dtype=np.int32)
        S = np.empty(self.n, dtype=np.int32)
        r = Result(hubs.ctypes.data_as(ctypes.POINTER(c_i32)), S.ctypes.data_as(ctypes.POINTER(c_i32)))
        check(lib().usaphmp_solve(self.h, generations, seed, ctypes.byref(r)))
        return {"hubs": hubs, "S": S, "cost_fp64": r.cost_fp64, "cost_fp32": r.cost_fp32,
                "evals": r.evals, "ms": r.ms}

    # step-level calls (device pointers)
    def initial_dev(self, mask_ptr, hubs_ptr, stream=0):
        check(lib().usaphmp_initial_dev(self.h, mask_ptr, hubs_ptr, stream))

    def children_dev(self, R, P, anc_ptr, seed, g, mask_ptr, hubs_ptr, stream=0):
        check(lib().usaphmp_children_dev(self.h, R, P, anc_ptr, seed, g, mask_ptr, hubs_ptr, stream))

    def allocate_dev(self, B, hubs_ptr, slot_ptr, stream=0):
        check(lib().usaphmp_allocate_dev(self.h, B, hubs_ptr, slot_ptr, stream))

    def eval_slots_dev(self, B, hubs_ptr, slot_ptr, fitness_ptr, stream=0):
        check(lib().usaphmp_eval_slots_dev(self.h, B, hubs_ptr, slot_ptr, fitness_ptr, stream))

    def select_dev(self, R, P, g, mask_ptr, fit_ptr, anc_ptr, anc_fit_ptr, best_ptr, best_fit_ptr, stream=0):
        check(lib().usaphmp_select_dev(self.h, R, P, g, mask_ptr, fit_ptr, anc_ptr, anc_fit_ptr, best_ptr,
                                       best_fit_ptr, stream))

    def local_search_dev(self, B, hubs_ptr, slot_ptr, max_sweeps, moves_ptr=None, sweeps_ptr=None, stream=0):
        check(lib().usaphmp_local_search_dev(self.h, B, hubs_ptr, slot_ptr, max_sweeps, moves_ptr, sweeps_ptr,
                                             stream))

    def rescore_fp64_dev(self, B, hubs_ptr, slot_ptr, cost_ptr, stream=0):
        check(lib().usaphmp_rescore_fp64_dev(self.h, B, hubs_ptr, slot_ptr, cost_ptr, stream))

    def ga_begin(self, seed, stream=0):
        check(lib().usaphmp_ga_begin(self.h, seed, stream))

    def ga_run(self, generations, stream=0):
        check(lib().usaphmp_ga_run(self.h, generations, stream))

    def ga_run_profiled(self, generations, stream=0):
        """Runs generations eagerly; returns {stage: summed device ms}."""
        acc = (c_f64 * 6)()
        check(lib().usaphmp_ga_run_profiled(self.h, generations, stream, acc))
        return dict(zip(STAGES, list(acc)))

    def ga_save(self, stream=0):
        """usaphmp_ga_save: the GA state as bytes."""
        nb = c_i64()
        check(lib().usaphmp_ga_state_bytes(self.h, ctypes.byref(nb)))
        buf = ctypes.create_string_buffer(nb.value)
        check(lib().usaphmp_ga_save(self.h, buf, nb.value, stream))
        return buf.raw

    def ga_load(self, state, stream=0):
        """usaphmp_ga_load: continue from a saved state."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        check(lib().usaphmp_ga_load(self.h, buf, len(state), stream))

    def ga_islands(self, stream=0):
        """usaphmp_ga_islands: (masks uint32 [R, nw], fitness float32 [R])."""
        R = self.params["islands"]
        masks = np.empty((R, self.nw), dtype=np.uint32)
        fit = np.empty(R, dtype=np.float32)
        check(lib().usaphmp_ga_islands(self.h, _ptr(masks), _ptr(fit), stream))
        return masks, fit

    def ga_population(self, stream=0):
        """usaphmp_ga_population: the last generation's children (masks uint32
        [R*P, nw]) and their raw fitness (float32 [R*P])."""
        prm = self.params
        B = prm["islands"] * prm["island_size"]
        masks = np.empty((B, self.nw), dtype=np.uint32)
        fit = np.empty(B, dtype=np.float32)
        check(lib().usaphmp_ga_population(self.h, _ptr(masks), _ptr(fit), stream))
        return masks, fit

    def ga_merge(self, mask, fit, stream=0):
        """usaphmp_ga_merge: every island's ancestor <- mask (uint32 [nw])."""
        mask = np.ascontiguousarray(mask, dtype=np.uint32)
        if mask.shape != (self.nw,):
            raise ValueError("mask must hold nw words")
        check(lib().usaphmp_ga_merge(self.h, _ptr(mask), float(fit), stream))

    def ga_result(self, stream=0):
        hubs = np.empty(self.p, dtype=np.int32)
        S = np.empty(self.n, dtype=np.int32)
        r = Result(hubs.ctypes.data_as(ctypes.POINTER(c_i32)), S.ctypes.data_as(ctypes.POINTER(c_i32)))
        check(lib().usaphmp_ga_result(self.h, ctypes.byref(r), stream))
        return {"hubs": hubs, "S": S, "cost_fp64": r.cost_fp64, "cost_fp32": r.cost_fp32, "evals": r.evals}


class Server:
    """Continuous-batching serving loop (a ``usaphmp_server_t``)."""

    def __init__(self, hbm_budget_bytes, max_active=32, path=PATH_SPLIT_BF16):
        h = c_vp()
        check(lib().usaphmp_server_create(int(hbm_budget_bytes), max_active, path, ctypes.byref(h)))
        self.h = h
        self._shape = {}

    def submit(self, W, C, p, chi=3.0, alpha=0.75, delta=2.0, islands=8, island_size=64, generations=200,
               seed=0):
        W = np.ascontiguousarray(W, dtype=np.float32)
        C = np.ascontiguousarray(C, dtype=np.float32)
        t = c_i64()
        check(lib().usaphmp_server_submit(self.h, W.shape[0], p, _ptr(W), _ptr(C), chi, alpha, delta, islands,
                                          island_size, generations, seed, ctypes.byref(t)))
        self._shape[t.value] = (W.shape[0], p)
        return t.value

    def step(self):
        a, q = c_i32(), c_i32()
        check(lib().usaphmp_server_step(self.h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def cancel(self, ticket):
        """usaphmp_server_cancel."""
        check(lib().usaphmp_server_cancel(self.h, ticket))

    def poll(self, ticket):
        """None while running; the result dict once finished (raises on failure)."""
        n, p = self._shape[ticket]
        hubs = np.empty(p, dtype=np.int32)
        S = np.empty(n, dtype=np.int32)
        r = Result(hubs.ctypes.data_as(ctypes.POINTER(c_i32)), S.ctypes.data_as(ctypes.POINTER(c_i32)))
        rc = lib().usaphmp_server_poll(self.h, ticket, ctypes.byref(r))
        if rc == 0:
            return None
        del self._shape[ticket]
        check(0 if rc == 1 else rc)
        return {"hubs": hubs, "S": S, "cost_fp64": r.cost_fp64, "cost_fp32": r.cost_fp32, "evals": r.evals,
                "ms": r.ms}

    def stats(self):
        """usaphmp_server_stats as a dict."""
        st = ServerStats()
        check(lib().usaphmp_server_stats(self.h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    @staticmethod
    def footprint(n, p, islands, island_size):
        b = c_i64()
        check(lib().usaphmp_server_footprint(n, p, islands, island_size, ctypes.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "h", None):
            lib().usaphmp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

"""Thin ctypes binding of libgmacop.so (include/gmacop.h): argument marshalling only.

Every step of the colony runs in the library's sm_103a kernels. There is no CPU fallback: importing
works without a GPU, but creating a Context raises if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_NO_ROUTE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_BUFFER, ERR_STATE = range(9)
THRESHOLD_OFF = 0xFFFFFFFF
FLAG_RANDOM_TAU = 1
FLAG_ANT_LOG = 2
FLAG_KERNEL_TIMING = 4
FLAG_NO_GRAPH = 8
FLAG_NO_LOCKSTEP = 16
MODE_AUTO, MODE_ITERATIVE, MODE_PERSISTENT = 0, 1, 2

_LIB = None


class Params(C.Structure):
    _fields_ = [("max_steps", C.c_uint32), ("h_sat_ms", C.c_uint32), ("thr_permille", C.c_uint32),
                ("flags", C.c_uint32), ("t_dep_ms", C.c_uint32), ("lanes_per_ant", C.c_uint32),
                ("mode", C.c_uint32), ("reserved", C.c_uint32)]


class Query(C.Structure):
    _fields_ = [("src", C.c_uint32), ("dst", C.c_uint32), ("n_ants", C.c_uint32), ("n_iter", C.c_uint32),
                ("alpha", C.c_float), ("beta", C.c_float), ("rho", C.c_float), ("reserved", C.c_uint32),
                ("seed", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("route", C.POINTER(C.c_uint32)), ("route_cap", C.c_uint32), ("route_len", C.c_uint32),
                ("travel_ms", C.c_uint64), ("wait_ms", C.c_uint64), ("ant_steps", C.c_uint64),
                ("n_success", C.c_uint64), ("best_iter", C.c_uint32), ("best_ant", C.c_uint32),
                ("status", C.c_int32), ("reserved", C.c_uint32)]


# name -> (restype, argtypes); the same names as include/gmacop.h
_vp, _u32, _u64, _f32, _i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_float, C.c_int
SIGNATURES = {
    "gmp_create": (_i32, [C.POINTER(_vp), _i32, _u64, _vp]),
    "gmp_destroy": (None, [_vp]),
    "gmp_strerror": (C.c_char_p, [_i32]),
    "gmp_last_error": (C.c_char_p, [_vp]),
    "gmp_set_stream": (_i32, [_vp, _vp]),
    "gmp_load_graph": (_i32, [_vp, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gmp_set_signals": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "gmp_set_red_times": (_i32, [_vp, _vp]),
    "gmp_set_densities": (_i32, [_vp, _vp]),
    "gmp_set_densities_async": (_i32, [_vp, _vp]),
    "gmp_set_params": (_i32, [_vp, C.POINTER(Params)]),
    "gmp_get_params": (_i32, [_vp, C.POINTER(Params)]),
    "gmp_solve": (_i32, [_vp, _u32, _u32, _u32, _u32, _f32, _f32, _f32, _u64, C.POINTER(Result)]),
    "gmp_solve_batch": (_i32, [_vp, _u32, C.POINTER(Query), C.POINTER(Result)]),
    "gmp_batch_stage": (_i32, [_vp, _u32, C.POINTER(Query)]),
    "gmp_batch_launch": (_i32, [_vp]),
    "gmp_batch_collect": (_i32, [_vp, C.POINTER(Result)]),
    "gmp_get_pheromone": (_i32, [_vp, _u32, _vp]),
    "gmp_get_ant_log": (_i32, [_vp, _u32, _vp, _u64]),
    "gmp_get_phase_order": (_i32, [_vp, _vp]),
    "gmp_get_edge_times": (_i32, [_vp, _vp, _vp]),
    "gmp_get_kernel_times": (_i32, [_vp, _vp]),
    "gmp_get_launch_count": (_i32, [_vp, C.POINTER(_u64)]),
    "gmp_solve_static": (_i32, [_vp, _u32, _u32, _u32, _u32, _f32, _f32, _f32, _u64, _vp, _vp, _u32]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgmacop.so; raises if it has not been built (no silent fallback)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libgmacop.so is not built ({path}); run paper_2010_14244_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


class GmpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{lib().gmp_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def _p(a):
    return None if a is None else a.ctypes.data


class Context:
    """One GPU + one road graph; wraps a gmp_ctx."""

    def __init__(self, device: int = 0, mem_budget: int = 0, stream=None):
        self._h = C.c_void_p()
        handle = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        rc = lib().gmp_create(C.byref(self._h), device, mem_budget, handle)
        if rc != OK:
            raise GmpError(rc, "gmp_create failed (is a CUDA device present?)")
        self.n_nodes = self.n_edges = 0
        self._queries = []

    def close(self):
        if self._h:
            lib().gmp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise GmpError(rc, lib().gmp_last_error(self._h).decode())

    def set_stream(self, stream=None):
        handle = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        self._check(lib().gmp_set_stream(self._h, handle))

    # ---------------------------------------------------------------- inputs
    def load_graph(self, net):
        a = dict(row_ptr=np.ascontiguousarray(net.row_ptr, np.uint32), col=np.ascontiguousarray(net.col, np.uint32),
                 length=np.ascontiguousarray(net.length_dm, np.uint32),
                 speed=np.ascontiguousarray(net.speed_kmh, np.uint16),
                 lanes=np.ascontiguousarray(net.lanes, np.uint8), x=np.ascontiguousarray(net.x_dm, np.int32),
                 y=np.ascontiguousarray(net.y_dm, np.int32))
        n, e = a["row_ptr"].size - 1, a["col"].size
        self._check(lib().gmp_load_graph(self._h, n, e, _p(a["row_ptr"]), _p(a["col"]), _p(a["length"]),
                                         _p(a["speed"]), _p(a["lanes"]), _p(a["x"]), _p(a["y"])))
        self.n_nodes, self.n_edges = n, e

    def set_signals(self, sig):
        a = [np.ascontiguousarray(sig.n_phases, np.uint8), np.ascontiguousarray(sig.cycle_ms, np.uint32),
             np.ascontiguousarray(sig.offset_ms, np.uint32), np.ascontiguousarray(sig.green_ms, np.uint32),
             np.ascontiguousarray(sig.edge_phase, np.uint8)]
        self._check(lib().gmp_set_signals(self._h, *(_p(x) for x in a)))

    def set_red_times(self, red_ms):
        r = np.ascontiguousarray(red_ms, np.uint32).reshape(-1)
        self._check(lib().gmp_set_red_times(self._h, _p(r)))

    def set_densities(self, vehicles):
        v = np.ascontiguousarray(vehicles, np.uint32)
        self._check(lib().gmp_set_densities(self._h, _p(v)))

    def set_densities_device(self, dev_ptr: int):
        self._check(lib().gmp_set_densities_async(self._h, C.c_void_p(dev_ptr)))

    def load_workload(self, wl):
        self.load_graph(wl.net)
        self.set_signals(wl.signals)
        self.set_densities(wl.vehicles)

    def set_params(self, max_steps=0, h_sat_ms=0, thr_permille=THRESHOLD_OFF, flags=0, t_dep_ms=0,
                   lanes_per_ant=0, mode=MODE_AUTO):
        p = Params(max_steps, h_sat_ms, thr_permille, flags, t_dep_ms, lanes_per_ant, mode, 0)
        self._check(lib().gmp_set_params(self._h, C.byref(p)))

    def get_params(self) -> dict:
        p = Params()
        self._check(lib().gmp_get_params(self._h, C.byref(p)))
        return {f: getattr(p, f) for f, _ in Params._fields_}

    # ---------------------------------------------------------------- solving
    @staticmethod
    def _cq(q) -> Query:
        return Query(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, 0, q.seed)

    def stage(self, queries):
        arr = (Query * len(queries))(*[self._cq(q) for q in queries])
        self._check(lib().gmp_batch_stage(self._h, len(queries), arr))
        self._queries = list(queries)

    def launch(self):
        self._check(lib().gmp_batch_launch(self._h))

    def collect(self, route_cap=None) -> list[dict]:
        n = len(self._queries)
        cap = (self.n_nodes + 1) if route_cap is None else route_cap
        bufs = [np.zeros(max(cap, 1), np.uint32) for _ in range(n)]
        res = (Result * n)()
        for i in range(n):
            res[i].route = bufs[i].ctypes.data_as(C.POINTER(C.c_uint32))
            res[i].route_cap = cap
        self._check(lib().gmp_batch_collect(self._h, res))
        return [self._result(res[i], bufs[i]) for i in range(n)]

    @staticmethod
    def _result(r: Result, buf) -> dict:
        return dict(status=r.status, route_len=r.route_len, travel_ms=r.travel_ms, wait_ms=r.wait_ms,
                    ant_steps=r.ant_steps, n_success=r.n_success, best_iter=r.best_iter, best_ant=r.best_ant,
                    route=buf[: r.route_len].copy() if r.status == OK else np.zeros(0, np.uint32))

    def solve_batch(self, queries, route_cap=None) -> list[dict]:
        n = len(queries)
        cap = (self.n_nodes + 1) if route_cap is None else route_cap
        arr = (Query * n)(*[self._cq(q) for q in queries])
        bufs = [np.zeros(max(cap, 1), np.uint32) for _ in range(n)]
        res = (Result * n)()
        for i in range(n):
            res[i].route = bufs[i].ctypes.data_as(C.POINTER(C.c_uint32))
            res[i].route_cap = cap
        self._check(lib().gmp_solve_batch(self._h, n, arr, res))
        self._queries = list(queries)
        return [self._result(res[i], bufs[i]) for i in range(n)]

    def solve(self, src, dst, n_ants, n_iter, alpha=1.0, beta=2.0, rho=0.1, seed=0, route_cap=None) -> dict:
        cap = (self.n_nodes + 1) if route_cap is None else route_cap
        buf = np.zeros(max(cap, 1), np.uint32)
        r = Result()
        r.route = buf.ctypes.data_as(C.POINTER(C.c_uint32))
        r.route_cap = cap
        rc = lib().gmp_solve(self._h, src, dst, n_ants, n_iter, alpha, beta, rho, seed, C.byref(r))
        if rc not in (OK, ERR_NO_ROUTE, ERR_BUFFER):
            raise GmpError(rc, lib().gmp_last_error(self._h).decode())
        return self._result(r, buf)

    def solve_static(self, src, dst, n_ants, n_iter, alpha, beta, rho, seed, d_result: int, d_route: int,
                     route_cap: int):
        """gmp_solve_static: device pointers for the result row and the route; asynchronous."""
        self._check(lib().gmp_solve_static(self._h, src, dst, n_ants, n_iter, alpha, beta, rho, seed,
                                           C.c_void_p(d_result), C.c_void_p(d_route), route_cap))

    # ---------------------------------------------------------------- inspection
    def pheromone(self, slot=0) -> np.ndarray:
        out = np.zeros(self.n_edges, np.uint64)
        self._check(lib().gmp_get_pheromone(self._h, slot, _p(out)))
        return out

    def ant_log(self, slot=0) -> np.ndarray:
        q = self._queries[slot]
        out = np.zeros((q.n_iter, q.n_ants, 4), np.uint32)
        self._check(lib().gmp_get_ant_log(self._h, slot, _p(out), out.size))
        return out

    def phase_order(self) -> np.ndarray:
        out = np.zeros((self.n_nodes, 8), np.uint8)
        self._check(lib().gmp_get_phase_order(self._h, _p(out)))
        return out

    def edge_times(self):
        tt = np.zeros(self.n_edges, np.uint32)
        qd = np.zeros(self.n_edges, np.uint32)
        self._check(lib().gmp_get_edge_times(self._h, _p(tt), _p(qd)))
        return tt, qd

    def kernel_times(self) -> dict:
        out = np.zeros(5, np.float32)
        self._check(lib().gmp_get_kernel_times(self._h, _p(out)))
        return dict(construct=float(out[0]), evaporate=float(out[1]), best=float(out[2]), queue=float(out[3]),
                    job=float(out[4]))

    def launch_count(self) -> int:
        n = C.c_uint64()
        self._check(lib().gmp_get_launch_count(self._h, C.byref(n)))
        return int(n.value)

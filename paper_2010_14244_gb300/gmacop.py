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
FLAG_REPULSIVE = 32
FLAG_UNIT_DEPOSIT = 64
FLAG_EVAP_UNUSED = 128
FLAG_PAPER_LITERAL = FLAG_REPULSIVE | FLAG_UNIT_DEPOSIT | FLAG_EVAP_UNUSED
FLAG_EXACT_H = 256
MODE_AUTO, MODE_ITERATIVE, MODE_PERSISTENT = 0, 1, 2
TAU_AUTO, TAU_DENSE, TAU_SPARSE = 0, 1, 2

_LIB = None


class TuneResult(C.Structure):
    _fields_ = [("lanes_per_ant", C.c_uint32), ("mode", C.c_uint32), ("queue_chunk", C.c_uint32),
                ("lockstep", C.c_uint32), ("branches", C.c_uint32), ("from_cache", C.c_uint32),
                ("n_tried", C.c_uint32),
                ("best_ms", C.c_float), ("default_ms", C.c_float), ("bucket", C.c_uint32 * 4),
                ("handoff_moves", C.c_uint32)]


class ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_uint32), ("max_ants", C.c_uint32), ("max_iter", C.c_uint32),
                ("mem_budget_mib", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_uint32), ("in_flight", C.c_uint32), ("busy_slots", C.c_uint32),
                ("done_waiting", C.c_uint32), ("jobs", C.c_uint64), ("completed", C.c_uint64),
                ("rejected", C.c_uint64)]


class Params(C.Structure):
    _fields_ = [("max_steps", C.c_uint32), ("h_sat_ms", C.c_uint32), ("thr_permille", C.c_uint32),
                ("flags", C.c_uint32), ("t_dep_ms", C.c_uint32), ("lanes_per_ant", C.c_uint32),
                ("mode", C.c_uint32), ("queue_chunk", C.c_uint32), ("branches", C.c_uint32),
                ("tau_layout", C.c_uint32), ("poll_limit", C.c_uint32), ("level_limit", C.c_uint32),
                ("handoff_moves", C.c_uint32)]


class Query(C.Structure):
    _fields_ = [("src", C.c_uint32), ("dst", C.c_uint32), ("n_ants", C.c_uint32), ("n_iter", C.c_uint32),
                ("alpha", C.c_float), ("beta", C.c_float), ("rho", C.c_float), ("reserved", C.c_uint32),
                ("seed", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("route", C.POINTER(C.c_uint32)), ("route_cap", C.c_uint32), ("route_len", C.c_uint32),
                ("travel_ms", C.c_uint64), ("wait_ms", C.c_uint64), ("ant_steps", C.c_uint64),
                ("n_success", C.c_uint64), ("best_iter", C.c_uint32), ("best_ant", C.c_uint32),
                ("status", C.c_int32), ("reserved", C.c_uint32)]


class Served(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("t_submit_ns", C.c_uint64), ("t_launch_ns", C.c_uint64),
                ("t_done_ns", C.c_uint64), ("clock_ms", C.c_uint64), ("slot", C.c_uint32),
                ("batch_size", C.c_uint32), ("result", Result)]


# name -> (restype, argtypes); the same names as include/gmacop.h
_vp, _u32, _u64, _f32, _i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_float, C.c_int
SIGNATURES = {
    "gmp_create": (_i32, [C.POINTER(_vp), _i32, _u64, _vp]),
    "gmp_destroy": (None, [_vp]),
    "gmp_strerror": (C.c_char_p, [_i32]),
    "gmp_last_error": (C.c_char_p, [_vp]),
    "gmp_set_stream": (_i32, [_vp, _vp]),
    "gmp_bind_workspace": (_i32, [_vp, _vp, _u64]),
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
    "gmp_get_densities": (_i32, [_vp, _vp]),
    "gmp_get_red_times": (_i32, [_vp, _vp]),
    "gmp_tick": (_i32, [_vp, _u64, _u32]),
    "gmp_autotune": (_i32, [_vp, _u32, C.POINTER(Query), _u32, C.POINTER(TuneResult)]),
    "gmp_autotune_reset": (None, []),
    "gmp_batch_reserve": (_i32, [_vp, _u32, _u64, _u32]),
    "gmp_multi_create": (_i32, [C.POINTER(_vp), _i32]),
    "gmp_multi_destroy": (None, [_vp]),
    "gmp_multi_last_error": (C.c_char_p, [_vp]),
    "gmp_multi_launch": (_i32, [_vp, C.POINTER(_vp), _u32]),
    "gmp_batch_ready": (_i32, [_vp, C.POINTER(C.c_int)]),
    "gmp_server_create": (_i32, [C.POINTER(_vp), _vp, _u32, C.POINTER(ServerConfig)]),
    "gmp_server_destroy": (None, [_vp]),
    "gmp_server_last_error": (C.c_char_p, [_vp]),
    "gmp_server_memory": (_i32, [_vp, C.POINTER(_u64), C.POINTER(_u64)]),
    "gmp_share_graph": (_i32, [_vp, _vp, C.c_int]),
    "gmp_server_submit": (_i32, [_vp, C.POINTER(Query), _u64]),
    "gmp_server_tick": (_i32, [_vp, _u64, _u32]),
    "gmp_server_pump": (_i32, [_vp, C.POINTER(ServerStats)]),
    "gmp_server_take": (_i32, [_vp, _u32, C.POINTER(Served), _vp, _u64, C.POINTER(_u32)]),
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

    def share_graph(self, owner, own_state: bool = False):
        """gmp_share_graph: read owner's road graph in place (and its traffic state, unless own_state)."""
        self._check(lib().gmp_share_graph(self._h, owner._h, int(bool(own_state))))
        self.n_nodes, self.n_edges = owner.n_nodes, owner.n_edges

    def bind_workspace(self, dev_ptr: int, nbytes: int):
        """gmp_bind_workspace: carve every later device allocation of this context from caller-owned
        device memory (e.g. tensor.data_ptr() of a uint8 CUDA tensor kept alive until close())."""
        self._check(lib().gmp_bind_workspace(self._h, C.c_void_p(dev_ptr) if dev_ptr else None, nbytes))

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
                   lanes_per_ant=0, mode=MODE_AUTO, queue_chunk=0, branches=0, tau_layout=TAU_AUTO, poll_limit=0,
                   level_limit=0, handoff_moves=0):
        p = Params(max_steps, h_sat_ms, thr_permille, flags, t_dep_ms, lanes_per_ant, mode, queue_chunk, branches,
                   tau_layout, poll_limit, level_limit, handoff_moves)
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

    def densities(self) -> np.ndarray:
        out = np.zeros(self.n_edges, np.uint32)
        self._check(lib().gmp_get_densities(self._h, _p(out)))
        return out

    def red_times(self) -> np.ndarray:
        out = np.zeros((self.n_nodes, 8), np.uint32)
        self._check(lib().gmp_get_red_times(self._h, _p(out)))
        return out

    def tick(self, t_now_ms: int, dt_ms: int):
        """gmp_tick: advance the traffic state by dt_ms at clock t_now_ms (asynchronous)."""
        self._check(lib().gmp_tick(self._h, t_now_ms, dt_ms))

    def autotune(self, probe_queries, probe_iter=0) -> dict:
        """gmp_autotune: time the schedules on a probe job (or reuse the bucket's cached choice) and
        apply the fastest to this context."""
        arr = (Query * len(probe_queries))(*[self._cq(q) for q in probe_queries])
        r = TuneResult()
        self._check(lib().gmp_autotune(self._h, len(probe_queries), arr, probe_iter, C.byref(r)))
        out = {f: getattr(r, f) for f, _ in TuneResult._fields_ if f != "bucket"}
        out["bucket"] = list(r.bucket)
        return out

    @staticmethod
    def autotune_reset():
        lib().gmp_autotune_reset()

    def reserve(self, n_queries: int, total_ants: int, max_iter: int):
        self._check(lib().gmp_batch_reserve(self._h, n_queries, total_ants, max_iter))

    def ready(self) -> bool:
        r = C.c_int()
        self._check(lib().gmp_batch_ready(self._h, C.byref(r)))
        return bool(r.value)

    def edge_times(self):
        tt = np.zeros(self.n_edges, np.uint32)
        qd = np.zeros(self.n_edges, np.uint32)
        self._check(lib().gmp_get_edge_times(self._h, _p(tt), _p(qd)))
        return tt, qd

    def kernel_times(self) -> dict:
        out = np.zeros(5, np.float32)
        self._check(lib().gmp_get_kernel_times(self._h, _p(out)))
        return dict(construct=float(out[0]), iter_end=float(out[1]), init_finalize=float(out[2]),
                    job=float(out[4]))

    def launch_count(self) -> int:
        n = C.c_uint64()
        self._check(lib().gmp_get_launch_count(self._h, C.byref(n)))
        return int(n.value)


class Server:
    """gmp_server: continuous batching over n_slots slots that share the road graph and traffic state of
    one context (`graph`, which must outlive the server)."""

    def __init__(self, graph, n_slots: int, max_batch: int, max_ants: int, max_iter: int, mem_budget_mib: int = 0):
        self.graph = graph
        cfg = ServerConfig(max_batch, max_ants, max_iter, mem_budget_mib)
        self._h = C.c_void_p()
        rc = lib().gmp_server_create(C.byref(self._h), graph._h, n_slots, C.byref(cfg))
        if rc != OK:
            raise GmpError(rc, lib().gmp_last_error(graph._h).decode())
        self.route_cap = graph.n_nodes + 1
        self._buf = np.zeros(1 << 16, np.uint32)
        self._out = (Served * 256)()

    def close(self):
        if self._h:
            lib().gmp_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise GmpError(rc, lib().gmp_server_last_error(self._h).decode())

    def memory(self) -> tuple[int, int]:
        """(bytes the slots' workspaces hold together, the server's budget in bytes; 0 = none)."""
        held, budget = _u64(), _u64()
        self._check(lib().gmp_server_memory(self._h, C.byref(held), C.byref(budget)))
        return int(held.value), int(budget.value)

    def submit(self, q, tag: int):
        cq = Context._cq(q)
        self._check(lib().gmp_server_submit(self._h, C.byref(cq), tag))

    def tick(self, t_now_ms: int, dt_ms: int):
        self._check(lib().gmp_server_tick(self._h, t_now_ms, dt_ms))

    def pump(self) -> dict:
        st = ServerStats()
        self._check(lib().gmp_server_pump(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def take(self) -> list[dict]:
        out = []
        while True:
            n = _u32()
            rc = lib().gmp_server_take(self._h, len(self._out), self._out, _p(self._buf), self._buf.size, C.byref(n))
            if rc == ERR_BUFFER:
                self._buf = np.zeros(self._buf.size * 4, np.uint32)
                continue
            self._check(rc)
            base = self._buf.ctypes.data
            for i in range(n.value):
                s = self._out[i]
                r = s.result
                off = (C.cast(r.route, C.c_void_p).value - base) // 4 if r.route else 0
                route = self._buf[off:off + r.route_len].copy() if r.status == OK else np.zeros(0, np.uint32)
                out.append(dict(tag=s.tag, t_submit_ns=s.t_submit_ns, t_launch_ns=s.t_launch_ns,
                                t_done_ns=s.t_done_ns, clock_ms=s.clock_ms, slot=s.slot, batch_size=s.batch_size,
                                status=r.status, route_len=r.route_len, travel_ms=r.travel_ms, wait_ms=r.wait_ms,
                                ant_steps=r.ant_steps, n_success=r.n_success, best_iter=r.best_iter,
                                best_ant=r.best_ant, route=route))
            if n.value == 0:
                return out


class Multi:
    """gmp_multi: the staged batches of several contexts (one road graph each) in one launch."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        rc = lib().gmp_multi_create(C.byref(self._h), device)
        if rc != OK:
            raise GmpError(rc, "gmp_multi_create failed")

    def close(self):
        if self._h:
            lib().gmp_multi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch(self, contexts):
        arr = (_vp * len(contexts))(*[c._h.value for c in contexts])
        rc = lib().gmp_multi_launch(self._h, arr, len(contexts))
        if rc != OK:
            raise GmpError(rc, lib().gmp_multi_last_error(self._h).decode())

    def solve(self, contexts, batches, route_cap=None) -> list[list[dict]]:
        """Stage batches[i] on contexts[i], launch all in one go, collect every context's results."""
        for c, qs in zip(contexts, batches):
            c.stage(qs)
        self.launch(contexts)
        return [c.collect(route_cap) for c in contexts]

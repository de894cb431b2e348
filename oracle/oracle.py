"""ctypes front end of the CPU oracle (oracle/orc_gmacop.c) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may use it.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIB = None

THR_OFF = 0xFFFFFFFF
FLAG_RANDOM_TAU = 1
FLAG_REPULSIVE = 32
FLAG_UNIT_DEPOSIT = 64
FLAG_EVAP_UNUSED = 128
FLAG_PAPER_LITERAL = FLAG_REPULSIVE | FLAG_UNIT_DEPOSIT | FLAG_EVAP_UNUSED
FLAG_EXACT_H = 256
ANT_SUCCESS, ANT_DEAD_END, ANT_STEP_CAP, ANT_TIME_CAP = 0, 1, 2, 3
OK, ERR_INVALID, ERR_NO_ROUTE, ERR_OOM, ERR_UNSUPPORTED, ERR_BUFFER = 0, 1, 2, 3, 6, 7


class _Net(C.Structure):
    _fields_ = [("n_nodes", C.c_uint32), ("n_edges", C.c_uint32)] + [
        (name, C.c_void_p)
        for name in ("row_ptr", "col", "length_dm", "speed_kmh", "lanes", "x_dm", "y_dm", "n_phases", "cycle_ms",
                     "offset_ms", "green_ms", "edge_phase", "vehicles", "red_ms")
    ]


class _Params(C.Structure):
    _fields_ = [("max_steps", C.c_uint32), ("h_sat_ms", C.c_uint32), ("thr_permille", C.c_uint32),
                ("flags", C.c_uint32), ("t_dep_ms", C.c_uint32), ("reserved", C.c_uint32)]


class _Query(C.Structure):
    _fields_ = [("src", C.c_uint32), ("dst", C.c_uint32), ("n_ants", C.c_uint32), ("n_iter", C.c_uint32),
                ("alpha", C.c_float), ("beta", C.c_float), ("rho", C.c_float), ("reserved", C.c_uint32),
                ("seed", C.c_uint64)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("route_len", C.c_uint32), ("travel_ms", C.c_uint64),
                ("wait_ms", C.c_uint64), ("ant_steps", C.c_uint64), ("n_success", C.c_uint64),
                ("best_iter", C.c_uint32), ("best_ant", C.c_uint32)]


@dataclass
class Params:
    max_steps: int = 0
    h_sat_ms: int = 0
    thr_permille: int = THR_OFF
    flags: int = 0
    t_dep_ms: int = 0

    def c(self) -> _Params:
        return _Params(self.max_steps, self.h_sat_ms, self.thr_permille, self.flags, self.t_dep_ms, 0)


def lib():
    global _LIB
    if _LIB is None:
        # ORC_LIB names a library built from a modified copy of the source (the planted-mistake tests)
        path = os.environ.get("ORC_LIB") or _build.build()
        L = C.CDLL(path)
        u32, u64, f32, vp = C.c_uint32, C.c_uint64, C.c_float, C.c_void_p
        sig = {
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_isqrt64": (u64, [u64]),
            "orc_free_flow_ms": (u32, [u32, u32]),
            "orc_capacity": (u32, [u32, u32]),
            "orc_edge_time_ms": (u32, [u32, u32, u32]),
            "orc_queue_delay_ms": (u32, [u32, u32, u32, C.c_int]),
            "orc_phase_order": (None, [u32, vp, vp, vp, u32, vp]),
            "orc_queue_preempt": (C.c_int, [vp, vp, vp]),
            "orc_signal_wait_ms": (u32, [u64, u32, u32, vp, vp, u32, u32]),
            "orc_kappa": (u64, [u32]),
            "orc_heuristic_ms": (u32, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, u64]),
            "orc_score": (f32, [u64, u32, u32, u32]),
            "orc_score_f": (f32, [u64, u32, u32, u32, u32]),
            "orc_tau_factor": (f32, [u64, u32]),
            "orc_log2": (f32, [f32]),
            "orc_exp2": (f32, [f32]),
            "orc_score_frac": (f32, [u64, f32, u32, f32, u32]),
            "orc_frac_constants": (None, [vp]),
            "orc_quantize": (None, [u32, vp, vp]),
            "orc_roulette_pick": (u32, [u32, vp, u64]),
            "orc_rho_fix": (u64, [f32]),
            "orc_evaporate": (u64, [u64, u64]),
            "orc_init_tau": (None, [u32, u64, u32, vp]),
            "orc_prepare": (C.c_int, [vp, vp, u32, vp, vp, vp, vp, vp, vp]),
            "orc_walk_one": (C.c_int, [vp, vp, vp, vp, u32, u32, vp, vp, vp, vp, vp]),
            "orc_solve": (C.c_int, [vp, vp, vp, vp, u32, vp, vp, vp]),
            "orc_tick": (C.c_int, [vp, vp, u64, u32, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------------------------- scalars
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return tuple(int(v) for v in o)


def isqrt(n: int) -> int:
    return int(lib().orc_isqrt64(n))


def free_flow_ms(length_dm, speed_kmh):
    return int(lib().orc_free_flow_ms(length_dm, speed_kmh))


def capacity(lanes, length_dm):
    return int(lib().orc_capacity(lanes, length_dm))


def edge_time_ms(ff, cap, n):
    return int(lib().orc_edge_time_ms(ff, cap, n))


def queue_delay_ms(n, h_sat_ms, lanes, signalised):
    return int(lib().orc_queue_delay_ms(n, h_sat_ms, lanes, int(bool(signalised))))


def signal_wait_ms(arr, cycle, offset, green, order, n_phases, phase):
    g = np.zeros(8, np.uint32)
    g[: len(green)] = green
    o = np.arange(8, dtype=np.uint8)
    o[: len(order)] = order
    return int(lib().orc_signal_wait_ms(arr, cycle, offset, _p(g), _p(o), n_phases, phase))


def phase_order(n_phases, Q, Th, red, T_max):
    q = np.zeros(8, np.uint64)
    q[:n_phases] = Q
    th = np.zeros(8, np.uint64)
    th[:n_phases] = Th
    r = np.zeros(8, np.uint32)
    r[:n_phases] = red
    out = np.zeros(8, np.uint8)
    lib().orc_phase_order(n_phases, _p(q), _p(th), _p(r), T_max, _p(out))
    return [int(v) for v in out[:n_phases]]


def kappa(v_max_kmh):
    return int(lib().orc_kappa(v_max_kmh))


def heuristic_ms(x, y, xd, yd, kap):
    return int(lib().orc_heuristic_ms(x, y, xd, yd, kap))


def score(tau, alpha, c_ms, beta, flags=None) -> np.float32:
    if flags is None:
        return np.float32(lib().orc_score(tau, alpha, c_ms, beta))
    return np.float32(lib().orc_score_f(tau, alpha, c_ms, beta, flags))


def tau_factor(tau, flags=0) -> np.float32:
    return np.float32(lib().orc_tau_factor(tau, flags))


def log2f(x) -> np.float32:
    return np.float32(lib().orc_log2(float(x)))


def exp2f(x) -> np.float32:
    return np.float32(lib().orc_exp2(float(x)))


def score_frac(tau, alpha, c_ms, beta, flags=0) -> np.float32:
    return np.float32(lib().orc_score_frac(tau, float(alpha), c_ms, float(beta), flags))


def frac_constants() -> np.ndarray:
    out = np.zeros(14, np.float32)
    lib().orc_frac_constants(_p(out))
    return out


def quantize(scores) -> np.ndarray:
    s = np.ascontiguousarray(scores, dtype=np.float32)
    w = np.zeros(s.size, np.uint64)
    lib().orc_quantize(s.size, _p(s), _p(w))
    return w


def roulette_pick(w, rnd):
    a = np.ascontiguousarray(w, dtype=np.uint64)
    return int(lib().orc_roulette_pick(a.size, _p(a), rnd))


def rho_fix(rho):
    return int(lib().orc_rho_fix(rho))


def evaporate(tau, rfix):
    return int(lib().orc_evaporate(tau, rfix))


def init_tau(n_edges, seed, flags=0):
    t = np.zeros(n_edges, np.uint64)
    lib().orc_init_tau(n_edges, seed, flags, _p(t))
    return t


# ---------------------------------------------------------------------------------------------- networks
class Net:
    """Keeps the numpy arrays alive behind the C struct."""

    def __init__(self, net, signals, vehicles, red_ms=None):
        self.arrays = dict(
            row_ptr=np.ascontiguousarray(net.row_ptr, np.uint32),
            col=np.ascontiguousarray(net.col, np.uint32),
            length_dm=np.ascontiguousarray(net.length_dm, np.uint32),
            speed_kmh=np.ascontiguousarray(net.speed_kmh, np.uint16),
            lanes=np.ascontiguousarray(net.lanes, np.uint8),
            x_dm=np.ascontiguousarray(net.x_dm, np.int32),
            y_dm=np.ascontiguousarray(net.y_dm, np.int32),
            n_phases=np.ascontiguousarray(signals.n_phases, np.uint8),
            cycle_ms=np.ascontiguousarray(signals.cycle_ms, np.uint32),
            offset_ms=np.ascontiguousarray(signals.offset_ms, np.uint32),
            green_ms=np.ascontiguousarray(signals.green_ms, np.uint32),
            edge_phase=np.ascontiguousarray(signals.edge_phase, np.uint8),
            vehicles=np.ascontiguousarray(vehicles, np.uint32),
            red_ms=None if red_ms is None else np.ascontiguousarray(red_ms, np.uint32),
        )
        self.n_nodes = int(net.row_ptr.shape[0] - 1)
        self.n_edges = int(net.col.shape[0])
        self.c = _Net(self.n_nodes, self.n_edges, *(_p(self.arrays[f[0]]) for f in _Net._fields_[2:]))

    @classmethod
    def from_workload(cls, wl, red_ms=None):
        return cls(wl.net, wl.signals, wl.vehicles, red_ms)


def _query(q) -> _Query:
    return _Query(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, 0, q.seed)


def prepare(net: Net, params: Params, dst: int) -> dict:
    E, N = net.n_edges, net.n_nodes
    out = {k: np.zeros(E, np.uint32) for k in ("ff", "cap", "tt", "qd")}
    out["h"] = np.zeros(N, np.uint32)
    out["order"] = np.zeros((N, 8), np.uint8)
    pr = params.c()
    rc = lib().orc_prepare(C.addressof(net.c), C.addressof(pr), dst, _p(out["ff"]), _p(out["cap"]),
                           _p(out["tt"]), _p(out["qd"]), _p(out["h"]), _p(out["order"]))
    if rc != OK:
        raise RuntimeError(f"orc_prepare failed: {rc}")
    return out


def queue_preempt(net: Net, params: Params | None = None) -> np.ndarray:
    order = np.zeros((net.n_nodes, 8), np.uint8)
    pr = (params or Params()).c()
    rc = lib().orc_queue_preempt(C.addressof(net.c), C.addressof(pr), _p(order))
    if rc != OK:
        raise RuntimeError(f"orc_queue_preempt failed: {rc}")
    return order


def tick(net: Net, params: Params, t_now: int, dt: int, order):
    """One serving tick: returns (vehicles, red_ms N x 8, new order N x 8)."""
    o = np.ascontiguousarray(order, np.uint8).reshape(-1)
    veh = np.zeros(net.n_edges, np.uint32)
    red = np.zeros((net.n_nodes, 8), np.uint32)
    new_order = np.zeros((net.n_nodes, 8), np.uint8)
    pr = params.c()
    rc = lib().orc_tick(C.addressof(net.c), C.addressof(pr), t_now, dt, _p(o), _p(veh), _p(red), _p(new_order))
    if rc != OK:
        raise RuntimeError(f"orc_tick failed: {rc}")
    return veh, red, new_order


def walk_one(net: Net, params: Params, query, tau, it=0, ant=0):
    """One ant: its status, route (roads; ``steps`` of them), moves (forward and back), T and W."""
    tau = np.ascontiguousarray(tau, np.uint64)
    route = np.zeros(max(2 * net.n_nodes, params.max_steps, 4096) + 1, np.uint32)  # >= the move cap
    steps, moves, T, W = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint32()
    pr, q = params.c(), _query(query)
    st = lib().orc_walk_one(C.addressof(net.c), C.addressof(pr), C.addressof(q), _p(tau), it, ant, _p(route),
                            C.byref(steps), C.byref(moves), C.byref(T), C.byref(W))
    if st < 0:
        raise ValueError(f"orc_walk_one rejected the query: {-st}")
    return dict(status=st, route_edges=route[: steps.value].copy(), steps=steps.value, moves=moves.value, T=T.value,
                W=W.value)


def log_fields(log):
    """Split an ant log (..., 4) into (status, roads in the route, moves, T, W) arrays."""
    log = np.asarray(log)
    w0 = log[..., 0].astype(np.uint32)
    return w0 & 0xFF, w0 >> 8, log[..., 1], log[..., 2], log[..., 3]


def solve(net: Net, params: Params, query, route_cap=None, want_tau=True, want_log=False) -> dict:
    cap = net.n_nodes + 1 if route_cap is None else route_cap
    route = np.zeros(max(cap, 1), np.uint32)
    tau = np.zeros(net.n_edges, np.uint64) if want_tau else None
    log = np.zeros((query.n_iter, query.n_ants, 4), np.uint32) if want_log else None
    res = _Result()
    pr, q = params.c(), _query(query)
    lib().orc_solve(C.addressof(net.c), C.addressof(pr), C.addressof(q), _p(route), cap, _p(tau), _p(log),
                    C.byref(res))
    out = dict(status=res.status, route_len=res.route_len, travel_ms=res.travel_ms, wait_ms=res.wait_ms,
               ant_steps=res.ant_steps, n_success=res.n_success, best_iter=res.best_iter, best_ant=res.best_ant)
    out["route"] = route[: res.route_len].copy() if res.status == OK else np.zeros(0, np.uint32)
    if want_tau:
        out["tau"] = tau
    if want_log:
        out["log"] = log
    return out


def solve_workload_query(wl, qi: int, params: Params | None = None, want_tau=True) -> dict:
    """Solve query ``qi`` of a workload (a top-level function so a spawned process pool can run it)."""
    net = Net.from_workload(wl)
    return solve(net, params or Params(), wl.queries[qi], want_tau=want_tau)

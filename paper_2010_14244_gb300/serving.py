"""Serving loop on the C ABI: Poisson route requests, periodic traffic ticks, continuous batching.

The loop only marshals: arrivals are submitted to the native server (gmp_server_*), which admits them
into jobs on idle slots; ticks advance the device-resident traffic state the slots share; finished
requests are taken back with their host timestamps. Latency is measured from each request's scheduled
arrival time to the moment the server saw its job finish (both on the host's monotonic clock).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import gmacop as G
from .workloads import Query


def make_server(wl, n_slots: int, max_batch: int, max_ants: int, max_iter: int, mem_budget: int = 0,
                device: int = 0, params: dict | None = None, tune_probe=None, tune_iter: int = 8):
    """A context holding the workload's road graph and traffic state, and a server of n_slots slots over it
    (the slots share that graph; mem_budget bounds their workspaces together, in bytes). Returns (server,
    [graph context]); the context must be closed after the server. On failure the context is closed
    before the error propagates. With tune_probe (requests shaped like a typical job), the autotuner picks
    the slots' schedule on that probe, tune_iter iterations, before the server starts; every schedule
    gives the same results."""
    graph = G.Context(device)
    try:
        graph.load_workload(wl)
        if params:
            graph.set_params(**params)
        if tune_probe:
            graph.autotune(list(tune_probe), probe_iter=tune_iter)
        return G.Server(graph, n_slots, max_batch, max_ants, max_iter, mem_budget >> 20), [graph]
    except Exception:
        graph.close()
        raise


@dataclass
class ServeReport:
    offered_per_s: float
    window_s: float
    submitted: int
    completed: int
    latencies_ms: np.ndarray = field(repr=False)
    ant_steps: int
    jobs: int
    ticks: int
    mean_batch: float
    routed: int = 0          # completed requests that found a route
    ant_walks: int = 0       # ants x iterations of the completed requests
    successes: int = 0       # ant walks that reached the destination
    unfinished: int = 0      # requests of the window still queued or running when the drain ended
    served_in_window: int = 0  # requests (of any arrival time) that finished inside the window
    window_only_s: float = 0.0  # length of the window alone
    results: list = field(repr=False, default_factory=list)

    def summary(self) -> dict:
        lat = self.latencies_ms
        per_s = (lambda n: n / self.window_s) if self.window_s else (lambda n: 0.0)
        return {
            "offered_req_per_s": self.offered_per_s,
            "window_s": self.window_s,
            "submitted": self.submitted,
            "completed": self.completed,
            "unfinished": self.unfinished,
            "queries_per_s": per_s(self.completed),
            "served_per_s_in_window": self.served_in_window / self.window_only_s if self.window_only_s else 0.0,
            "routed_queries_per_s": per_s(self.routed),
            "routed_fraction": self.routed / self.completed if self.completed else 0.0,
            "success_fraction": self.successes / self.ant_walks if self.ant_walks else 0.0,
            "ant_steps_per_s": per_s(self.ant_steps),
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_batch": self.mean_batch,
            "jobs": self.jobs,
            "ticks": self.ticks,
        }


def uniform_requests(n_nodes: int, n_ants: int, n_iter: int, seed: int = 0):
    """Uniform origin-destination requests (src != dst), seeded; the request's own seed is its index."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def make(i: int) -> Query:
        s = int(rng.integers(n_nodes))
        d = int(rng.integers(n_nodes - 1))
        d += d >= s
        return Query(s, d, n_ants, n_iter, 1.0, 2.0, 0.1, 1_000_003 * i + seed)

    return make


def run_poisson(server: G.Server, make_request, rate_per_s: float, duration_s: float, warmup_s: float = 0.0,
                tick_ms: int = 1000, clock_start_ms: int = 0, seed: int = 0, drain_s: float = 30.0,
                keep_results: bool = False) -> ServeReport:
    """Offer Poisson arrivals at rate_per_s for warmup_s + duration_s seconds, tick the traffic state
    every tick_ms of wall time, and report the requests that arrived inside the measured window."""
    rng = np.random.Generator(np.random.PCG64(seed + 17))
    total = warmup_s + duration_s
    t0 = time.perf_counter_ns()
    arrivals: dict[int, int] = {}  # tag -> scheduled arrival (ns, monotonic)
    walks: dict[int, int] = {}     # tag -> ants x iterations
    next_arr = rng.exponential(1.0 / rate_per_s)
    next_tick = tick_ms / 1000.0
    clock = clock_start_ms
    tag = 0
    ticks = 0
    done: list[dict] = []
    deadline = total + drain_s
    while True:
        now = (time.perf_counter_ns() - t0) * 1e-9
        while next_arr <= now and next_arr < total:
            q = make_request(tag)
            arrivals[tag] = t0 + int(next_arr * 1e9)
            walks[tag] = q.n_ants * q.n_iter
            server.submit(q, tag)
            tag += 1
            next_arr += rng.exponential(1.0 / rate_per_s)
        if now >= next_tick and now < total:
            server.tick(clock, tick_ms)
            clock += tick_ms
            ticks += 1
            next_tick += tick_ms / 1000.0
        st = server.pump()
        done.extend(server.take())
        if now >= total and st["queued"] == 0 and st["in_flight"] == 0 and st["done_waiting"] == 0:
            break
        if now >= deadline:
            break
    w0 = t0 + int(warmup_s * 1e9)
    w1 = t0 + int(total * 1e9)
    win = [r for r in done if w0 <= arrivals[r["tag"]] < w1]
    lat = np.array([(r["t_done_ns"] - arrivals[r["tag"]]) * 1e-6 for r in win], np.float64)
    last_done = max((r["t_done_ns"] for r in win), default=w1)
    window = (max(w1, last_done) - w0) * 1e-9
    submitted = sum(1 for a in arrivals.values() if w0 <= a < w1)
    return ServeReport(offered_per_s=rate_per_s, window_s=window, submitted=submitted, completed=len(win),
                       latencies_ms=lat, ant_steps=int(sum(r["ant_steps"] for r in win)),
                       jobs=int(st["jobs"]), ticks=ticks,
                       mean_batch=float(np.mean([r["batch_size"] for r in win])) if win else 0.0,
                       routed=sum(1 for r in win if r["status"] == 0),
                       ant_walks=sum(walks[r["tag"]] for r in win),
                       successes=int(sum(r["n_success"] for r in win)), unfinished=submitted - len(win),
                       served_in_window=sum(1 for r in done if w0 <= r["t_done_ns"] < w1),
                       window_only_s=(w1 - w0) * 1e-9, results=done if keep_results else [])

#!/usr/bin/env python
"""Throughput of the MACO-P route colony on GB300: ant-steps/s and routed queries/s.

Workload (one "step"): the 64x64 perturbed-grid road network (4096 intersections, 14,916 directed roads,
2-phase signals at every node, 2000 Zipf(1.2) vehicles), 16 origin-destination colonies x 1024 ants x 200
iterations, alpha=1, beta=2, rho=0.1, run as one device job (construction, evaporation+deposit, best
tracking and the queue/preemption update every iteration). Every launch starts from fresh pheromone, so
each step repeats identical work with identical, oracle-checked results.

  python bench.py [--steps K] [--warmup W] [--gpus N]        # the CUDA library
  python bench.py --impl reference ...                       # the CPU oracle on the host cores

Under torchrun each rank runs an independent replica (colonies are independent problems: weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6772.9
# DRAM bytes (read + write) of one construction launch of this workload's kernel and schedule, from an ncu
# capture of the current kernel (one chain's launch of 1024 walks, alone and with cold caches): the graph
# and the pheromone tables stay in L2, so DRAM carries the cold start only. Set to None when the kernel
# changes, until it is captured again.
CONSTRUCT_TRAFFIC_BYTES = 803_072


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gmacop", choices=["gmacop", "reference"])
    p.add_argument("--mode", type=int, default=0, help="0 auto, 1 iterative, 2 persistent")
    p.add_argument("--lanes", type=int, default=0, help="lanes per ant (0 = autotune)")
    p.add_argument("--free-running", action="store_true",
                   help="with --lanes/--mode: sub-warp ants without warp lockstep (the tuner's pick for grid64)")
    p.add_argument("--handoff", type=int, default=0,
                   help="with --lanes/--mode: hand walks longer than this many moves to the tail kernel")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the one-colony-per-launch comparison")
    p.add_argument("--no-serving", action="store_true", help="skip the serving legs and the geo100k job")
    p.add_argument("--iterations", type=int, default=0, help="override iterations (profiling runs only)")
    p.add_argument("--queries", type=int, default=0, help="override colony count (profiling runs only)")
    return p.parse_args()


_OVERRIDE = {}


def workload():
    from paper_2010_14244_gb300 import workloads

    wl = workloads.grid64()
    if _OVERRIDE.get("iterations"):
        for q in wl.queries:
            q.n_iter = _OVERRIDE["iterations"]
    if _OVERRIDE.get("queries"):
        wl.queries = wl.queries[: _OVERRIDE["queries"]]
    return wl


def workload_config(wl):
    q = wl.queries[0]
    return {"workload": f"grid64: 64x64 perturbed grid, {wl.net.n_nodes} nodes, {wl.net.n_edges} directed roads, "
                        f"{len(wl.queries)} OD colonies x {q.n_ants} ants x {q.n_iter} iterations",
            "nodes": wl.net.n_nodes, "roads": wl.net.n_edges, "colonies": len(wl.queries), "ants": q.n_ants,
            "iterations": q.n_iter, "alpha": q.alpha, "beta": q.beta, "rho": q.rho}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int) -> float:
    """The largest value over the ranks (the slowest rank's time); NCCL ranks reduce on their GPU."""
    if world <= 1:
        return x
    import torch

    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------ CPU oracle
_WL = None
_WL_NAME = None


def _make_workload(name):
    from paper_2010_14244_gb300 import workloads

    if name == "grid64":
        return workload()
    if name == "geo100k":
        return workloads.geo100k()
    if name == "city_batch":
        return workloads.city_batch()
    if name == "geo1m":
        return workloads.geo1m_serving()
    raise ValueError(name)


def _pool_init(name="grid64"):
    global _WL, _WL_NAME
    _WL_NAME = name
    _WL = _make_workload(name)


def _pool_query(item):
    """item: a colony index; (graph, colony) for the city batch; ("req", i) for a serving request."""
    if _WL_NAME == "city_batch":
        g, qi = item
        return _WL[g], _WL[g].queries[qi]
    if _WL_NAME == "geo1m":  # request i of the serving stream (the stream draws its pairs in order)
        from paper_2010_14244_gb300 import serving

        make = serving.uniform_requests(_WL.net.n_nodes, SERVE_ANTS, SERVE_ITERS, seed=9)
        return _WL, [make(j) for j in range(item[1] + 1)][-1]
    return _WL, _WL.queries[item]


_ONETS = {}


def _pool_solve(item):
    from oracle import oracle as orc

    wl, q = _pool_query(item)
    if id(wl) not in _ONETS:
        _ONETS[id(wl)] = orc.Net.from_workload(wl)
    r = orc.solve(_ONETS[id(wl)], orc.Params(), q, want_tau=False)
    return r["ant_steps"], r["status"], r["n_success"], q.n_ants * q.n_iter


def oracle_run(pool, items):
    t0 = time.perf_counter()
    out = pool.map(_pool_solve, items, chunksize=1)
    dt = time.perf_counter() - t0
    return out, dt


def make_pool(name="grid64", want=16):
    import multiprocessing as mp

    cores = min(len(os.sched_getaffinity(0)), want)
    return mp.get_context("spawn").Pool(cores, initializer=_pool_init, initargs=(name,)), cores


def _one_core_solve(item):
    t0 = time.perf_counter()
    steps, status, *_ = _pool_solve(item)
    return steps, status, time.perf_counter() - t0


def oracle_baseline(name, items, what):
    """The oracle as it stands on the host cores, on a bounded sample of a workload: one warm-up pass (the
    workers build the workload and load the oracle), then the timed pass, one colony per process."""
    pool, cores = make_pool(name, len(items))
    try:
        oracle_run(pool, items[:cores])  # warm-up: workers build the workload and load the library
        out, dt = oracle_run(pool, items)
        one_steps, _, one_dt = pool.apply(_one_core_solve, (items[0],))
    finally:
        pool.close()
        pool.join()
    steps = sum(o[0] for o in out)
    routed = sum(o[1] == 0 for o in out)
    return {"value": steps / dt, "unit": "ant-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{what}: {len(items)} colonies, one per process over {cores} processes, after a warm-up "
                      f"pass; {dt:.1f} s wall",
            "queries_per_s": len(items) / dt, "routed_queries_per_s": routed / dt,
            "success_fraction": sum(o[2] for o in out) / max(1, sum(o[3] for o in out)),
            "one_core": {"value": one_steps / one_dt, "unit": "ant-steps/s", "queries_per_s": 1.0 / one_dt,
                         "sample": f"the first colony of the sample alone in one process, {one_dt:.2f} s"}}


def cpu_baseline_line(n_queries):
    return oracle_baseline("grid64", list(range(n_queries)), f"all {n_queries} colonies of the workload, full size")


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workload()
    nq = len(wl.queries)
    pool, cores = make_pool()
    routed = 0
    try:
        for _ in range(args.warmup):
            oracle_run(pool, list(range(nq)))
        tot_steps, tot_t = 0, 0.0
        for _ in range(args.steps):
            out, dt = oracle_run(pool, list(range(nq)))
            tot_steps += sum(o[0] for o in out)
            routed += sum(o[1] == 0 for o in out)
            tot_t += dt
    finally:
        pool.close()
        pool.join()
    v = tot_steps / tot_t
    line = {"impl": "reference", "metric": "ant-steps/s", "value": v, "unit": "ant-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
            "data": "synthetic", "config": workload_config(wl),
            "queries_per_s": nq * args.steps / tot_t, "routed_queries_per_s": routed / tot_t,
            "cpu_baseline": {"value": v, "unit": "ant-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: all {nq} colonies at full size over {cores} processes"},
            "e2e": {"value": v, "unit": "ant-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------ legs
SERVE_SLOTS, SERVE_RATE, SERVE_WINDOW_S, SERVE_WARMUP_S, SERVE_MAX_BATCH = 16, 2000.0, 2.0, 0.5, 64
SERVE_1M_SLOTS = 8
SERVE_1M_SAT_S = 6.0  # window of the saturated 1M-node run: a job there takes a few hundred ms, so a short
                      # window counts too few completions to be steady
SERVE_ANTS, SERVE_ITERS = 128, 30
SERVE_TUNE_PROBE = 32  # requests in the probe job that picks the serving slots' schedule
SERVE_1M_TUNE_PROBE = 64


def bytes_per_ant_step(n_nodes, n_edges):
    """Algorithmic bytes of one construction step: the row bounds (8) and per candidate its 32-byte road
    record, its 8-byte pheromone/heuristic pair and the head's 16-byte signal window (d = E/N candidates),
    plus the route write (4): 12 + 56 d."""
    return 12.0 + 56.0 * n_edges / n_nodes


def routed_summary(results, queries, seconds):
    """Colonies that found a route per second, and what fraction of colonies and ant walks succeeded."""
    routed = int(sum(r["status"] == 0 for r in results))
    walks = sum(q.n_ants * q.n_iter for q in queries)
    return {"routed": routed, "routed_queries_per_s": routed / seconds, "routed_fraction": routed / max(1, len(results)),
            "success_fraction": sum(int(r["n_success"]) for r in results) / max(1, walks)}


def leg_roofline(bpa, steps, seconds, peak, peak_kind, what):
    achieved = bpa * steps / seconds / 1e9
    return {"bound": "hbm", "kernel": "construct", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": None, "bytes_per_ant_step": bpa,
            "time": what}


def timed_launches(launch, stream, n_warm=2, n_timed=3):
    """Median device time (ms) of a launch callable on `stream`, L2 flushed before each timed launch."""
    import torch

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    times = []
    with torch.cuda.stream(stream):
        for _ in range(n_warm):
            launch()
        stream.synchronize()
        for _ in range(n_timed):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def geo100k_leg(with_cpu):
    """The batched job on the 100k-node planar graph: 512 colonies x 256 ants x 100 iterations in one job
    (autotuned schedule; the sparse pheromone layout applies at this size)."""
    import torch

    from paper_2010_14244_gb300 import gmacop, workloads

    wl = workloads.geo100k()
    stream = torch.cuda.Stream()
    ctx = gmacop.Context(0, stream=stream)
    try:
        ctx.load_workload(wl)
        tune = ctx.autotune(wl.queries, probe_iter=8)
        ctx.stage(wl.queries)
        ms = timed_launches(ctx.launch, stream)
        res = ctx.collect()
    finally:
        ctx.close()
    steps = sum(r["ant_steps"] for r in res)
    peak, kind = peaks()
    out = {"workload": f"geo100k: 100k-node planar graph, {wl.net.n_edges} roads, 512 OD colonies x 256 ants x "
                       "100 iterations", "ms_per_job": ms, "ant_steps_per_job": steps,
           "ant_steps_per_s": steps / (ms / 1e3), "queries_per_s": len(res) / (ms / 1e3),
           **routed_summary(res, wl.queries, ms / 1e3),
           "roofline": leg_roofline(bytes_per_ant_step(wl.net.n_nodes, wl.net.n_edges), steps, ms / 1e3, peak, kind,
                                    "job device time, median of 3, L2 flushed"),
           "schedule": {k: tune[k] for k in ("lanes_per_ant", "mode", "branches", "lockstep", "handoff_moves")}}
    if with_cpu:
        out["cpu_baseline"] = oracle_baseline("geo100k", list(range(0, 512, 32)),
                                              "every 32nd colony of the same job, full size")
    return out


def city_batch_leg(with_cpu):
    """64 independent city graphs (1k-200k nodes) with all their colonies in one launch, 50 iterations."""
    import torch

    from paper_2010_14244_gb300 import gmacop, workloads

    cities = workloads.city_batch()
    streams = [torch.cuda.Stream() for _ in cities]  # one per context: their jobs overlap in the launch
    ctxs = []
    m = gmacop.Multi(0)
    try:
        for wl, st in zip(cities, streams):
            c = gmacop.Context(0, stream=st)
            c.load_workload(wl)
            c.stage(wl.queries)
            ctxs.append(c)
        # the launch runs after the work queued on every context's stream and before any later work on
        # them, so events on the first context's stream bracket it
        ms = timed_launches(lambda: m.launch(ctxs), streams[0])
        res = [c.collect() for c in ctxs]
    finally:
        m.close()
        for c in ctxs:
            c.close()
    flat = [r for rs in res for r in rs]
    queries = [q for wl in cities for q in wl.queries]
    steps = sum(r["ant_steps"] for r in flat)
    n_nodes = sum(wl.net.n_nodes for wl in cities)
    n_edges = sum(wl.net.n_edges for wl in cities)
    peak, kind = peaks()
    out = {"workload": f"city batch: 64 planar city graphs, {n_nodes} nodes, {n_edges} roads, {len(flat)} colonies "
                       "of 128-1024 ants x 50 iterations, one launch", "ms_per_job": ms, "ant_steps_per_job": steps,
           "ant_steps_per_s": steps / (ms / 1e3), "queries_per_s": len(flat) / (ms / 1e3),
           **routed_summary(flat, queries, ms / 1e3),
           "roofline": leg_roofline(bytes_per_ant_step(n_nodes, n_edges), steps, ms / 1e3, peak, kind,
                                    "job device time, median of 3, L2 flushed")}
    if with_cpu:
        items = [(g, 0) for g in range(0, 64, 4)]
        out["cpu_baseline"] = oracle_baseline("city_batch", items, "the first colony of every 4th city, full size")
    return out


def serving_leg_1m(with_cpu):
    """Route requests on a 1M-node planar road graph with 5M vehicles: uniform origin-destination pairs,
    128 ants x 30 iterations each, 1 s traffic ticks, 8 slots sharing the graph. First Poisson arrivals at
    20k req/s, far above what the GPU completes (each request is about 7 M ant-steps): the figure is the
    saturated throughput, requests finished per second inside the window whenever they arrived. Then
    arrivals at 70 % of that throughput, where the latency percentiles describe the service itself."""
    from paper_2010_14244_gb300 import serving, workloads

    wl = workloads.geo1m_serving()
    make = serving.uniform_requests(wl.net.n_nodes, SERVE_ANTS, SERVE_ITERS, seed=9)
    # the slots' schedule: the autotuner's choice on a probe job of 64 requests from the same stream (the
    # saturated run's jobs are large; a 32-request probe picked a schedule slower on them)
    probe = [make(i) for i in range(SERVE_1M_TUNE_PROBE)]
    srv, keep = serving.make_server(wl, n_slots=SERVE_1M_SLOTS, max_batch=128, max_ants=SERVE_ANTS,
                                    max_iter=SERVE_ITERS, tune_probe=probe)
    schedule = schedule_of(keep[0])
    try:
        sat = serving.run_poisson(srv, make, rate_per_s=20000.0, duration_s=SERVE_1M_SAT_S, warmup_s=1.0,
                                  tick_ms=1000, drain_s=0.0).summary()
    finally:
        srv.close()
        for c in keep:
            c.close()
    capacity = sat["served_per_s_in_window"]
    srv, keep = serving.make_server(wl, n_slots=SERVE_1M_SLOTS, max_batch=128, max_ants=SERVE_ANTS,
                                    max_iter=SERVE_ITERS, tune_probe=probe)
    try:
        make = serving.uniform_requests(wl.net.n_nodes, SERVE_ANTS, SERVE_ITERS, seed=9)
        rep = serving.run_poisson(srv, make, rate_per_s=max(1.0, 0.7 * capacity), duration_s=SERVE_WINDOW_S,
                                  warmup_s=SERVE_WARMUP_S, tick_ms=1000)
    finally:
        srv.close()
        for c in keep:
            c.close()
    out = rep.summary()
    peak, kind = peaks()
    out.update(slots=SERVE_1M_SLOTS, ants=SERVE_ANTS, iterations=SERVE_ITERS, arrivals="poisson, uniform OD",
               schedule=schedule, schedule_source=f"autotuned on a probe job of {SERVE_1M_TUNE_PROBE} requests",
               network=f"{wl.net.n_nodes} nodes, {wl.net.n_edges} roads, 5M vehicles",
               tick="1 s (queue/preemption update with vehicle discharge)",
               at_20k_offered={k: sat[k] for k in ("offered_req_per_s", "served_per_s_in_window", "submitted",
                                                     "unfinished", "ant_steps_per_s", "mean_batch")},
               roofline=leg_roofline(bytes_per_ant_step(wl.net.n_nodes, wl.net.n_edges), rep.ant_steps,
                                     rep.window_s, peak, kind, "serving window (wall time)"))
    if with_cpu:
        out["cpu_baseline"] = oracle_baseline("geo1m", [("req", i) for i in range(16)],
                                              "the first 16 requests of the stream, against the traffic at clock 0")
    return out


def serving_leg(wl):
    """Route requests on the same road network: Poisson arrivals with uniform origin-destination pairs,
    128 ants x 30 iterations each, traffic ticks every second, continuous batching over slot contexts."""
    from paper_2010_14244_gb300 import serving

    make = serving.uniform_requests(wl.net.n_nodes, SERVE_ANTS, SERVE_ITERS, seed=5)
    probe = [make(i) for i in range(SERVE_TUNE_PROBE)]  # the slots' schedule: autotuned on a probe job
    srv, slots = serving.make_server(wl, n_slots=SERVE_SLOTS, max_batch=SERVE_MAX_BATCH, max_ants=SERVE_ANTS,
                                     max_iter=SERVE_ITERS, tune_probe=probe)
    schedule = schedule_of(slots[0])
    try:
        make = serving.uniform_requests(wl.net.n_nodes, SERVE_ANTS, SERVE_ITERS, seed=5)
        rep = serving.run_poisson(srv, make, rate_per_s=SERVE_RATE, duration_s=SERVE_WINDOW_S,
                                  warmup_s=SERVE_WARMUP_S, tick_ms=1000)
    finally:
        srv.close()
        for c in slots:
            c.close()
    out = rep.summary()
    out.update(slots=SERVE_SLOTS, ants=SERVE_ANTS, iterations=SERVE_ITERS, arrivals="poisson, uniform OD",
               schedule=schedule, schedule_source=f"autotuned on a probe job of {SERVE_TUNE_PROBE} requests",
               tick="1 s (queue/preemption update with vehicle discharge)")
    return out


def schedule_of(ctx):
    """The schedule a context runs (the parameters the autotuner sets)."""
    p = ctx.get_params()
    return {k: p[k] for k in ("mode", "lanes_per_ant", "branches", "handoff_moves", "flags", "tau_layout")}


# ------------------------------------------------------------------------------------------ GPU
def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2010_14244_gb300 import gmacop

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    wl = workload()
    nq = len(wl.queries)
    ctx = gmacop.Context(local_rank, stream=stream)
    ctx.load_workload(wl)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # schedule: the autotuner's choice for this size bucket (timed on a 32-iteration probe of the same
    # colonies, not inside any timed region), unless the command line fixes one
    tune = None
    if args.lanes == 0 and args.mode == 0:
        tune = ctx.autotune(wl.queries, probe_iter=32)
    else:
        ctx.set_params(mode=args.mode, lanes_per_ant=args.lanes, handoff_moves=args.handoff,
                       flags=gmacop.FLAG_NO_LOCKSTEP if args.free_running else 0)
    sched = {k: v for k, v in ctx.get_params().items()
             if k in ("mode", "lanes_per_ant", "queue_chunk", "branches", "tau_layout", "flags", "handoff_moves")}

    def timed_region(flags):
        """K steps, each bracketed by CUDA events on the library's stream, L2 flushed in between."""
        ctx.set_params(**dict(sched, flags=sched["flags"] | flags))
        ctx.stage(wl.queries)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                ctx.launch()
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            times, kt = [], dict(construct=0.0, iter_end=0.0, init_finalize=0.0, job=0.0)
            for _ in range(args.steps):
                flush.zero_()  # L2 flush between timed steps (not timed)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.launch()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                if flags & gmacop.FLAG_KERNEL_TIMING:
                    for k, v in ctx.kernel_times().items():
                        kt[k] += v
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
        return times, kt

    # timed region 1: the job as users run it (the throughput figure)
    sampler = ClockSampler(local_rank)
    sampler.start()
    times, _ = timed_region(0)
    clocks = sampler.stop()
    res = ctx.collect()
    steps_per_job = sum(r["ant_steps"] for r in res)
    launches = ctx.launch_count()
    # timed region 2: the same job with event records around every kernel (per-kernel durations)
    times_k, kt = timed_region(gmacop.FLAG_KERNEL_TIMING)
    res2 = ctx.collect()
    assert [r["travel_ms"] for r in res2] == [r["travel_ms"] for r in res]
    total_ms = max_over_ranks(sum(times), world)

    # the job's critical path, from a per-ant log of the same job (not timed): iterations are synchronous,
    # so each colony takes at least the sum over iterations of its longest walk, one dependent step after
    # another; the slowest colony bounds the job
    ctx.set_params(**dict(sched, flags=sched["flags"] | gmacop.FLAG_ANT_LOG))
    ctx.solve_batch(wl.queries)
    longest = [int(ctx.ant_log(i)[:, :, 1].max(axis=1).sum()) for i in range(nq)]  # moves of the longest walk
    crit_steps = max(longest)
    slow = int(np.argmax(longest))
    # the slowest colony alone, as its own job in the same schedule (not timed with the rest): its walks are
    # the same as in the batch, so the batch costs job / alone times its own critical chain
    ctx.set_params(**sched)
    ctx.stage([wl.queries[slow]])
    alone = []
    with torch.cuda.stream(stream):
        ctx.launch()
        stream.synchronize()
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.launch()
            e1.record(stream)
            e1.synchronize()
            alone.append(e0.elapsed_time(e1))
    assert ctx.collect()[0]["travel_ms"] == res[slow]["travel_ms"]
    alone_ms = statistics.median(alone)
    critical = {"longest_walk_steps_summed_over_iterations": crit_steps, "colony": slow,
                "us_per_critical_step": (total_ms / args.steps) * 1e3 / crit_steps,
                "slowest_colony_alone_ms": alone_ms,
                "job_over_slowest_colony_alone": (total_ms / args.steps) / alone_ms,
                "how": "job device time / (max over colonies of the sum over iterations of the longest walk); "
                       "the slowest colony alone is its own job, same schedule, median of 3"}

    # the plain form: each colony its own job (stage, launch, collect), one after another
    plain = None
    if not args.no_plain:
        ctx.set_params(**sched)
        with torch.cuda.stream(stream):
            ctx.solve_batch(wl.queries[:1])  # warm (captures the one-colony job graph)
            stream.synchronize()
            t0 = time.perf_counter()
            plain_res = [ctx.solve_batch([q])[0] for q in wl.queries]
            plain_t = time.perf_counter() - t0
        plain_steps = sum(r["ant_steps"] for r in plain_res)
        plain = {"queries_per_s": nq / plain_t, "ant_steps_per_s": plain_steps / plain_t, "ms": plain_t * 1e3,
                 **routed_summary(plain_res, wl.queries, plain_t),
                 "how": f"the same {nq} colonies, each solved as its own job (stage, launch, collect) in sequence"}

    # end to end through the public API: densities and queries from pinned host memory, results back
    e2e = None
    if not args.no_e2e:
        veh = torch.from_numpy(wl.vehicles.astype(np.uint32)).pin_memory()
        veh_np = veh.numpy()
        e2e_t, e2e_steps, d2h, e2e_routed = 0.0, 0, 0, 0
        ctx.set_params(**sched)
        with torch.cuda.stream(stream):
            ctx.set_densities(veh_np)
            ctx.solve_batch(wl.queries)  # warm (captures the job graph)
            for _ in range(args.steps):
                flush.zero_()
                stream.synchronize()
                t0 = time.perf_counter()
                ctx.set_densities(veh_np)
                out = ctx.solve_batch(wl.queries)
                e2e_t += time.perf_counter() - t0
                e2e_steps += sum(r["ant_steps"] for r in out)
                e2e_routed += sum(r["status"] == gmacop.OK for r in out)
                d2h = nq * 48 + sum(4 * r["route_len"] for r in out)
        e2e = {"value": e2e_steps / e2e_t, "unit": "ant-steps/s",
               "h2d_bytes_per_step": int(wl.net.n_edges * 4 + nq * 40), "d2h_bytes_per_step": int(d2h),
               "queries_per_s": nq * args.steps / e2e_t, "routed_queries_per_s": e2e_routed / e2e_t}
    # the same colonies with the exact heuristic (a different colony, so not the headline): its job time,
    # ant-steps and routes next to the default straight-line bound's
    exact = None
    if not args.no_plain:
        ctx.set_params(**dict(sched, flags=sched["flags"] | gmacop.FLAG_EXACT_H))
        ctx.stage(wl.queries)
        ex_times = []
        with torch.cuda.stream(stream):
            for _ in range(2):
                ctx.launch()
            stream.synchronize()
            for _ in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.launch()
                e1.record(stream)
                e1.synchronize()
                ex_times.append(e0.elapsed_time(e1))
        rex = ctx.collect()
        ex_ms = statistics.median(ex_times)
        ex_steps = sum(r["ant_steps"] for r in rex)
        exact = {"ms_per_job": ex_ms, "ant_steps_per_job": ex_steps, "ant_steps_per_s": ex_steps / (ex_ms / 1e3),
                 "queries_per_s": nq / (ex_ms / 1e3), "successful_ants": int(sum(r["n_success"] for r in rex)),
                 "successful_ants_default": int(sum(r["n_success"] for r in res)),
                 "mean_best_travel_s": float(np.mean([r["travel_ms"] for r in rex]) / 1e3),
                 "mean_best_travel_s_default": float(np.mean([r["travel_ms"] for r in res]) / 1e3)}
        ctx.set_params(**sched)
    ctx.close()
    serving = serving_1m = geo = city = None
    with_cpu = world == 1 and not args.no_cpu_baseline
    if not args.no_serving and rank == 0:
        serving = serving_leg(wl)
        serving_1m = serving_leg_1m(with_cpu)
        geo = geo100k_leg(with_cpu)
        city = city_batch_leg(with_cpu)
    if rank != 0:
        return
    K = args.steps
    value = world * steps_per_job * K / (total_ms / 1e3)
    n, e = wl.net.n_nodes, wl.net.n_edges
    d = e / n
    bytes_per_step = 12 + 56 * d  # algorithmic bytes per ant-step of the construction kernel
    # the construction launches of the concurrent colony chains overlap in time, so the rate is the
    # job's algorithmic construction bytes over the job's device time (region 1): a lower bound on
    # the construction kernels' own rate (the iteration ends take part of that time)
    construct_launches = (launches - 2) // 2  # per job: init, result rows, and per chain iteration two
    achieved = bytes_per_step * steps_per_job * K / (total_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": "ant-steps/s", "value": value, "unit": "ant-steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
        "config": dict(workload_config(wl), l2="flushed between timed steps (256 MB write)",
                       schedule={k: sched[k] for k in ("mode", "lanes_per_ant", "queue_chunk", "branches",
                                                        "tau_layout", "handoff_moves")},
                       lockstep=None if tune is None else tune["lockstep"],
                       schedule_source="autotuned" if tune is not None else "command line"),
        "queries_per_s": world * nq * K / (total_ms / 1e3),
        **{k: (v * world if k == "routed_queries_per_s" else v)
           for k, v in routed_summary(res, wl.queries, total_ms / 1e3 / K).items()},
        "ant_steps_per_step": steps_per_job,
        "kernel_ms_per_step": {k: v / K for k, v in kt.items()},
        "ms_per_step_with_kernel_events": sum(times_k) / K,
        "roofline": {"bound": "hbm", "kernel": "construct (all colony chains)", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": CONSTRUCT_TRAFFIC_BYTES,
                     "traffic_scope": "DRAM bytes of one construction launch (ncu, one chain alone, cold caches; "
                                      "the tail kernel of a hand-off schedule reads about 0.88 MB more per launch)",
                     "algorithmic_bytes_per_launch": bytes_per_step * steps_per_job / max(construct_launches, 1),
                     "algorithmic_bytes_per_job": bytes_per_step * steps_per_job,
                     "bytes_per_ant_step": bytes_per_step,
                     "time": "job device time (construction launches of concurrent chains overlap)",
                     "construct_launches_per_job": construct_launches,
                     "avg_launch_ms_summed_over_chains": kt["construct"] / (K * max(construct_launches, 1)),
                     "binding_limit": "the dependent step chain of the slowest colony (critical_path), not HBM: "
                                      "the graph and pheromone tables are L2-resident"},
        "critical_path": critical,
        "gpu_launches": launches * K,
        "clocks": clocks,
    }
    if e2e:
        line["e2e"] = e2e
    if plain:
        line["plain_one_colony_per_launch"] = plain
    if tune is not None:
        line["autotune"] = {k: tune[k] for k in ("n_tried", "best_ms", "default_ms", "bucket")}
    if serving:
        line["serving"] = serving
    if serving_1m:
        line["serving_1m_nodes"] = serving_1m
    if geo:
        line["batched_geo100k"] = geo
    if city:
        line["batched_city_graphs"] = city
    if exact:
        line["exact_heuristic"] = exact
    if with_cpu:
        line["cpu_baseline"] = cpu_baseline_line(nq)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    _OVERRIDE.update(iterations=args.iterations, queries=args.queries)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch

        backend = "nccl" if args.impl == "gmacop" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

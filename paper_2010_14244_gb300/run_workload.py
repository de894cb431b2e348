"""Run one named workload through the library a few times (for timing and for profiler captures).

    python -m paper_2010_14244_gb300.run_workload grid64 --iterations 6 --repeat 2
    python -m paper_2010_14244_gb300.run_workload geo100k --queries 64 --iterations 4
    python -m paper_2010_14244_gb300.run_workload geo1m --queries 64 --ants 128 --iterations 30 --ticks 3
    python -m paper_2010_14244_gb300.run_workload grid64 --flags 256      # exact heuristic
    python -m paper_2010_14244_gb300.run_workload grid10 --mode 2 --lanes 8  # the persistent job

Prints one JSON line per run with the job's device time (CUDA events on the library's stream) and the
library's per-kernel-group times of that job with --kernel-times (construction, iteration end,
init + finalize, whole job).
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    p = argparse.ArgumentParser()
    p.add_argument("workload", choices=["grid10", "grid64", "geo100k", "geo1m"])
    p.add_argument("--queries", type=int, default=0, help="colonies (0 = the workload's own)")
    p.add_argument("--ants", type=int, default=0, help="ants per colony (0 = the workload's own)")
    p.add_argument("--iterations", type=int, default=0, help="iterations (0 = the workload's own)")
    p.add_argument("--repeat", type=int, default=2)
    p.add_argument("--ticks", type=int, default=0, help="serving ticks of 1 s before each run")
    p.add_argument("--lanes", type=int, default=0)
    p.add_argument("--mode", type=int, default=0)
    p.add_argument("--tau-layout", type=int, default=0)
    p.add_argument("--flags", type=int, default=0, help="GMP_FLAG_* bits (e.g. 256: exact heuristic)")
    p.add_argument("--kernel-times", action="store_true", help="events around every kernel; report their times")
    p.add_argument("--alpha", type=float, default=0.0, help="pheromone exponent of every colony (0 = its own)")
    p.add_argument("--free-running", action="store_true", help="sub-warp ants without warp lockstep")
    p.add_argument("--pheromone", action="store_true", help="read colony 0's pheromone table after each run")
    p.add_argument("--handoff", type=int, default=0,
                   help="hand walks longer than this many moves to the tail kernel (0 = off)")
    args = p.parse_args()

    import dataclasses

    import torch

    from . import build, gmacop, serving
    from . import workloads as W

    build.build()
    if args.workload == "grid10":
        wl = W.grid10()
    elif args.workload == "grid64":
        wl = W.grid64()
    elif args.workload == "geo100k":
        wl = W.geo100k(n_queries=args.queries or 512)
    else:
        wl = W.geo1m_serving()
        make = serving.uniform_requests(wl.net.n_nodes, args.ants or 128, args.iterations or 30, seed=9)
        wl.queries = [make(i) for i in range(args.queries or 64)]
    qs = wl.queries[: args.queries] if args.queries else wl.queries
    qs = [dataclasses.replace(q, n_ants=args.ants or q.n_ants, n_iter=args.iterations or q.n_iter,
                              alpha=args.alpha or q.alpha) for q in qs]
    stream = torch.cuda.Stream()
    ctx = gmacop.Context(0, stream=stream)
    ctx.load_workload(wl)
    flags = args.flags | (gmacop.FLAG_KERNEL_TIMING if args.kernel_times else 0)
    flags |= gmacop.FLAG_NO_LOCKSTEP if args.free_running else 0
    ctx.set_params(mode=args.mode, lanes_per_ant=args.lanes, tau_layout=args.tau_layout, flags=flags,
                   handoff_moves=args.handoff)
    ctx.stage(qs)
    clock = 0
    for r in range(args.repeat):
        for _ in range(args.ticks):
            ctx.tick(clock, 1000)
            clock += 1000
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            ctx.launch()
            e1.record(stream)
            e1.synchronize()
        res = ctx.collect()
        if args.pheromone:
            ctx.pheromone(0)
        print(json.dumps({"run": r, "workload": args.workload, "colonies": len(qs), "job_ms": e0.elapsed_time(e1),
                          "kernel_ms": ctx.kernel_times() if args.kernel_times else None,
                          "host_ms": (time.perf_counter() - t0) * 1e3,
                          "ant_steps": int(sum(x["ant_steps"] for x in res)),
                          "found": int(sum(x["status"] == 0 for x in res))}), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()

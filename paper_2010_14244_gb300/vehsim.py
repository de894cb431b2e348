"""Vehicle-level MACO-P loop (Fig. 3 over n vehicles) on top of the colony and the serving tick.

Every vehicle is either at a node, waiting to choose its next road, or between two nodes on a road it
has chosen (Fig. 3's vehicle between two nodes: it keeps going to that road's head). Time advances in steps
of dt (1 s). Per step at clock t:

  1. the roads' vehicle counts are the simulated vehicles on them (the traffic this experiment studies);
     they refresh the congested travel times, queue delays and phase orders (gmp_set_densities);
  2. every vehicle at a node that is not its destination asks the colony for a route from there to its
     destination departing at t; all of a step's requests run as one batched job, each colony keyed by
     (simulation seed, vehicle, decision) so a vehicle's choice depends only on it and the traffic state;
     the vehicle takes the first road of the best route (no route: it stays and asks again next step);
  3. a vehicle that takes road e reaches its head at t + tt_e and leaves it after the signal wait there
     (the approach's green window under the current phase order, plus the queue delay; none at its
     destination or at an unsignalised node): the same road model the colony scores with;
  4. vehicles whose road ends within the step stand at its head at the next step (or have arrived);
  5. gmp_tick(t, dt) advances the signals' red-time accumulators and phase orders by the step (the
     counts it discharges are replaced by the vehicles' own counts at the next step).

The experiment of Table 1 (overall travel time against the number of vehicles) is `run_table`; the
network is a synthetic stand-in of the paper's map (`workloads.city52`). The loop talks to the colony
through a small backend interface, implemented here over the library (`LibraryBackend`).
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W

AT_NODE, ON_ROAD, ARRIVED = 0, 1, 2


@dataclass
class SimConfig:
    dt_ms: int = 1000
    n_ants: int = 32
    n_iter: int = 8
    alpha: float = 1.0
    beta: float = 2.0
    rho: float = 0.1
    flags: int = 0
    max_time_ms: int = 4 * 3600 * 1000
    seed: int = 0


@dataclass
class SimReport:
    n_vehicles: int
    arrived: int
    makespan_s: float  # clock when the last vehicle arrived (the overall travel time of the fleet)
    mean_trip_s: float
    p50_trip_s: float
    p99_trip_s: float
    mean_signal_wait_s: float
    decisions: int  # colony solves (one per vehicle per node, plus retries)
    retries: int  # decisions that found no route
    steps: int
    wall_s: float
    trip_ms: np.ndarray = field(repr=False, default=None)
    path_edges: list = field(repr=False, default=None)

    def summary(self) -> dict:
        return {k: v for k, v in self.__dict__.items() if k not in ("trip_ms", "path_edges")}


class LibraryBackend:
    """The colony, road model and tick of one library context (gmacop.Context) on one graph."""

    def __init__(self, ctx, wl: W.Workload, flags: int = 0):
        self.ctx = ctx
        self.net = wl.net
        self.sig = wl.signals
        self.flags = flags
        ctx.load_graph(wl.net)
        ctx.set_signals(wl.signals)
        ctx.set_densities(np.zeros(wl.net.n_edges, np.uint32))
        ctx.set_red_times(np.zeros((wl.net.n_nodes, 8), np.uint32))

    def set_densities(self, veh: np.ndarray):
        self.ctx.set_densities(veh)

    def road_state(self):
        tt, qd = self.ctx.edge_times()
        return tt, qd, self.ctx.phase_order()

    def route_batch(self, t_ms: int, queries: list) -> list:
        self.ctx.set_params(t_dep_ms=t_ms, flags=self.flags)
        return [(r["status"], r["route"]) for r in self.ctx.solve_batch(queries)]

    def tick(self, t_ms: int, dt_ms: int):
        self.ctx.tick(t_ms, dt_ms)


def signal_wait(arr, cycle, offset, green, order, phase):
    """Wait at a signalised head for vehicles reaching the stop line at absolute times arr (arrays over
    vehicles; green and order are the head's 8-phase rows): 0 inside the approach's green window under
    the phase order, else the time to its next start (windows laid out in order from the offset)."""
    arr = np.asarray(arr, np.int64)
    cycle = np.asarray(cycle, np.int64)
    rows = np.arange(len(phase))
    pos = np.argmax(order == phase[:, None], axis=1)  # the approach phase's place in the order
    cum = np.cumsum(np.take_along_axis(green, order.astype(np.int64), axis=1), axis=1)
    glen = green[rows, phase]
    start = cum[rows, pos] - glen  # its window starts after the greens ordered before it
    c = (arr % cycle + cycle - np.asarray(offset, np.int64) % cycle) % cycle  # position in the cycle
    return np.where((c >= start) & (c < start + glen), 0, (start + cycle - c) % cycle)


class VehicleSim:
    def __init__(self, backend, cfg: SimConfig):
        self.b = backend
        self.cfg = cfg
        net = backend.net
        self.N, self.E = net.n_nodes, net.n_edges
        self.col = net.col.astype(np.int64)
        tails = net.tails().astype(np.int64)
        self.keys = tails * self.N + self.col  # sorted: CSR rows ascending, heads ascending within a row
        assert np.all(np.diff(self.keys) >= 0)
        sig = backend.sig
        self.nph = sig.n_phases.astype(np.int64)
        self.cycle = sig.cycle_ms.astype(np.int64)
        self.offset = sig.offset_ms.astype(np.int64)
        self.green = sig.green_ms.reshape(self.N, 8).astype(np.int64)
        self.ephase = sig.edge_phase.astype(np.int64)

    def edge_id(self, u: np.ndarray, v: np.ndarray) -> np.ndarray:
        k = u * self.N + v
        i = np.searchsorted(self.keys, k)
        assert np.all(self.keys[np.minimum(i, self.E - 1)] == k), "route step is not a road"
        return i

    def run(self, src, dst, depart_ms=None, keep_paths=False) -> SimReport:
        cfg = self.cfg
        src = np.asarray(src, np.int64)
        dst = np.asarray(dst, np.int64)
        n = src.size
        if n >= 1 << 20 or cfg.seed >= 1 << 24:
            raise ValueError("colony seeds pack (seed, vehicle, decision) into 24 + 20 + 20 bits")
        depart = np.zeros(n, np.int64) if depart_ms is None else np.asarray(depart_ms, np.int64)
        state = np.where(src == dst, ARRIVED, AT_NODE)
        node = src.copy()
        road = np.full(n, -1, np.int64)
        ready = depart.copy()  # at a node: from when it may choose; on a road: when it leaves the road's head
        arrive = np.where(src == dst, depart, -1)
        n_dec = np.zeros(n, np.int64)
        sig_wait = np.zeros(n, np.int64)
        paths = [[] for _ in range(n)] if keep_paths else None
        decisions = retries = steps = 0
        t = 0
        w0 = time.perf_counter()
        while np.any(state != ARRIVED) and t < cfg.max_time_ms:
            on = state == ON_ROAD
            veh = np.bincount(road[on], minlength=self.E).astype(np.uint32)
            self.b.set_densities(veh)
            deciding = np.flatnonzero((state == AT_NODE) & (ready <= t))
            if deciding.size:
                qs = [W.Query(int(node[i]), int(dst[i]), cfg.n_ants, cfg.n_iter, cfg.alpha, cfg.beta, cfg.rho,
                              (cfg.seed << 40) | (int(i) << 20) | int(n_dec[i] & 0xFFFFF)) for i in deciding]
                res = self.b.route_batch(t, qs)
                decisions += len(qs)
                n_dec[deciding] += 1
                ok = np.array([st == 0 and len(rt) > 1 for st, rt in res], bool)
                retries += int((~ok).sum())
                go = deciding[ok]
                if go.size:
                    nxt = np.array([int(rt[1]) for (st, rt), k in zip(res, ok) if k], np.int64)
                    e = self.edge_id(node[go], nxt)
                    tt, qd, order = self.b.road_state()
                    arr = t + tt[e].astype(np.int64)
                    wait = np.zeros(go.size, np.int64)
                    sgn = (nxt != dst[go]) & (self.nph[nxt] > 0)
                    if np.any(sgn):
                        h = nxt[sgn]
                        wait[sgn] = signal_wait(arr[sgn], self.cycle[h], self.offset[h], self.green[h],
                                                order[h].astype(np.int64), self.ephase[e[sgn]])
                        sig_wait[go[sgn]] += wait[sgn]
                        wait[sgn] += qd[e[sgn]].astype(np.int64)
                    state[go] = ON_ROAD
                    road[go] = e
                    node[go] = nxt
                    ready[go] = arr + wait
                    if keep_paths:
                        for i, ei in zip(go, e):
                            paths[i].append(int(ei))
            # roads that end within this step: the vehicle stands at the head (or has arrived)
            done = np.flatnonzero((state == ON_ROAD) & (ready <= t + cfg.dt_ms))
            fin = done[node[done] == dst[done]]
            arrive[fin] = ready[fin]
            state[fin] = ARRIVED
            road[fin] = -1
            mid = done[node[done] != dst[done]]
            state[mid] = AT_NODE
            road[mid] = -1
            self.b.tick(t, cfg.dt_ms)
            t += cfg.dt_ms
            steps += 1
        wall = time.perf_counter() - w0
        arrived = state == ARRIVED
        trip = np.where(arrived, arrive - depart, -1)
        tr = trip[arrived] / 1000.0
        return SimReport(n, int(arrived.sum()), float(arrive[arrived].max() / 1000.0) if arrived.any() else 0.0,
                         float(tr.mean()) if tr.size else 0.0, float(np.percentile(tr, 50)) if tr.size else 0.0,
                         float(np.percentile(tr, 99)) if tr.size else 0.0,
                         float(sig_wait[arrived].mean() / 1000.0) if arrived.any() else 0.0, decisions, retries, steps,
                         wall, trip, paths)


def fleet(n_nodes: int, n_vehicles: int, seed: int):
    """n uniform origin-destination pairs (origin != destination), all entering at clock 0."""
    pairs = W.uniform_od(n_nodes, n_vehicles, np.random.Generator(np.random.PCG64(seed)))
    return np.array([p[0] for p in pairs]), np.array([p[1] for p in pairs])


def run_table(ctx, counts, cfg: SimConfig | None = None, wl: W.Workload | None = None) -> list[dict]:
    """Table 1's experiment on the synthetic network: the fleet grows, each size is simulated to the end."""
    cfg = cfg or SimConfig()
    wl = wl or W.city52()
    rows = []
    for n in counts:
        be = LibraryBackend(ctx, wl, cfg.flags)
        src, dst = fleet(wl.net.n_nodes, n, seed=1000 + n)
        rep = VehicleSim(be, cfg).run(src, dst)
        rows.append(rep.summary())
    return rows


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--vehicles", default="300,600,900,1200,1500,1800,2100,2400,2700,3000,3300,3600,3900,4200,4500")
    p.add_argument("--ants", type=int, default=32)
    p.add_argument("--iterations", type=int, default=8)
    p.add_argument("--flags", type=int, default=0)
    args = p.parse_args()
    from . import build, gmacop

    build.build()
    ctx = gmacop.Context(0)
    try:
        cfg = SimConfig(n_ants=args.ants, n_iter=args.iterations, flags=args.flags)
        for row in run_table(ctx, [int(v) for v in args.vehicles.split(",")], cfg):
            print(json.dumps(row), flush=True)
    finally:
        ctx.close()


if __name__ == "__main__":
    main()

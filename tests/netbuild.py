"""Hand-built tiny road networks for tests (raw inputs only: topology, attributes, signals, vehicles)."""
from __future__ import annotations

import heapq

import numpy as np

from paper_2010_14244_gb300 import workloads as W


def build(n_nodes, roads, coords=None, signals=None, vehicles=None, bidirectional=True):
    """roads: list of (a, b, length_dm, speed_kmh[, lanes[, orient]]).
    signals: {node: (cycle_ms, offset_ms, [green per phase])}; approach phase of a road = its orient.
    vehicles: {(tail, head): count} on directed roads."""
    a = [r[0] for r in roads]
    b = [r[1] for r in roads]
    L = [r[2] for r in roads]
    v = [r[3] for r in roads]
    lanes = [r[4] if len(r) > 4 else 3 for r in roads]
    orient = [r[5] if len(r) > 5 else 0 for r in roads]
    if coords is None:
        coords = [(0, 0)] * n_nodes
    x = [c[0] for c in coords]
    y = [c[1] for c in coords]
    net = W.csr_from_roads(n_nodes, a, b, L, v, lanes, orient, x, y, bidirectional=bidirectional)
    n_ph = np.zeros(n_nodes, np.uint8)
    cyc = np.zeros(n_nodes, np.uint32)
    off = np.zeros(n_nodes, np.uint32)
    green = np.zeros((n_nodes, 8), np.uint32)
    for node, (c, o, g) in (signals or {}).items():
        n_ph[node] = len(g)
        cyc[node] = c
        off[node] = o
        green[node, : len(g)] = g
    sig = W.SignalTiming(n_ph, cyc, off, green.ravel(), net.orient.copy())
    veh = np.zeros(net.n_edges, np.uint32)
    tails = net.tails()
    for (t, h), n in (vehicles or {}).items():
        idx = np.flatnonzero((tails == t) & (net.col == h))
        assert idx.size == 1
        veh[idx[0]] = n
    return net, sig, veh


def edge_id(net, t, h):
    tails = net.tails()
    idx = np.flatnonzero((tails == t) & (net.col == h))
    assert idx.size == 1
    return int(idx[0])


class Timing:
    """Arrival-time function of each road built from the oracle's per-road primitives, which are
    pinned separately; used by the textbook searches below."""

    def __init__(self, orc, onet, net, sig, dst, params=None):
        self.orc = orc
        self.net = net
        self.sig = sig
        self.dst = dst
        self.t_dep = 0 if params is None else params.t_dep_ms
        self.prep = orc.prepare(onet, params or orc.Params(), dst)

    def after(self, e, t):
        """Elapsed time after taking road e when leaving its tail at elapsed time t; returns (t', wait)."""
        v = int(self.net.col[e])
        arr = t + int(self.prep["tt"][e])
        if v == self.dst or self.sig.n_phases[v] == 0:
            return arr, 0
        w = self.orc.signal_wait_ms(self.t_dep + arr, int(self.sig.cycle_ms[v]), int(self.sig.offset_ms[v]),
                                    [int(g) for g in self.sig.green_ms[v * 8: v * 8 + 8]],
                                    [int(o) for o in self.prep["order"][v]], int(self.sig.n_phases[v]),
                                    int(self.sig.edge_phase[e]))
        w += int(self.prep["qd"][e])
        return arr + w, w


def td_dijkstra(net, timing: Timing, src, dst):
    """Earliest arrival with FIFO arrival-time functions (label-setting Dijkstra on elapsed time)."""
    INF = float("inf")
    best = [INF] * net.n_nodes
    best[src] = 0
    pq = [(0, src)]
    done = [False] * net.n_nodes
    while pq:
        t, u = heapq.heappop(pq)
        if done[u]:
            continue
        done[u] = True
        if u == dst:
            return t
        for e in range(int(net.row_ptr[u]), int(net.row_ptr[u + 1])):
            v = int(net.col[e])
            t2, _ = timing.after(e, t)
            if t2 < best[v]:
                best[v] = t2
                heapq.heappush(pq, (t2, v))
    return None


def brute_force_min(net, timing: Timing, src, dst):
    """Minimum elapsed time over every simple path src -> dst (exhaustive DFS)."""
    best = [None]
    seen = {src}

    def dfs(u, t):
        if u == dst:
            if best[0] is None or t < best[0]:
                best[0] = t
            return
        for e in range(int(net.row_ptr[u]), int(net.row_ptr[u + 1])):
            v = int(net.col[e])
            if v in seen:
                continue
            seen.add(v)
            dfs(v, timing.after(e, t)[0])
            seen.discard(v)

    dfs(src, 0)
    return best[0]

"""The vehicle-level loop (Fig. 3 over n vehicles) on the oracle backend: its road-motion arithmetic
against the oracle's signal wait, a hand-worked trip, and fleet invariants (every vehicle arrives along
a valid walk, no trip is shorter than its free-flow shortest path, one decision per road taken plus the
retries). No GPU needed."""
import heapq

import numpy as np

from paper_2010_14244_gb300 import vehsim as V
from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
from tests.vehsim_oracle import OracleBackend


def test_host_signal_wait_equals_oracle(orc):
    rng = np.random.default_rng(2)
    for _ in range(400):
        P = int(rng.integers(2, 9))
        green = np.zeros(8, np.int64)
        green[:P] = rng.integers(0, 40000, P)
        green[int(rng.integers(0, P))] += 1000
        cycle = int(green.sum())
        offset = int(rng.integers(0, 3 * cycle))
        order = np.arange(8)
        order[:P] = rng.permutation(P)
        phase = int(rng.integers(0, P))
        arr = rng.integers(0, 2**31, 16)
        got = V.signal_wait(arr, np.full(16, cycle), np.full(16, offset), np.tile(green, (16, 1)),
                            np.tile(order, (16, 1)), np.full(16, phase))
        want = [orc.signal_wait_ms(int(a), cycle, offset, list(green[:P]), list(order[:P]), P, phase) for a in arr]
        assert list(got) == want


def _line():
    """0 - 1 - 2, node 1 signalised (cycle 20 s, phase 0 green [0, 8 s)), roads 45 km/h: 512 dm = 4096 ms."""
    roads = [(0, 1, 512, 45, 3, 0), (1, 2, 1024, 45, 3, 0)]
    net, sig, veh = NB.build(3, roads, [(0, 0), (512, 0), (1536, 0)], {1: (20000, 0, [8000, 12000])})
    return W.Workload("line", net, sig, veh)


def test_hand_worked_trip_on_a_line(orc):
    """Decide at node 0 at t = 0; reach node 1 at 4096 ms, inside phase 0's green: no wait, no queue;
    stand at node 1 from the step at 5000 ms, decide there; reach node 2 (the destination, no wait) after
    8192 ms: arrival at 13192 ms. Two decisions, one per road."""
    wl = _line()
    rep = V.VehicleSim(OracleBackend(orc, wl), V.SimConfig(n_ants=4, n_iter=2)).run([0], [2], keep_paths=True)
    assert rep.arrived == 1 and rep.decisions == 2 and rep.retries == 0
    assert int(rep.trip_ms[0]) == 5000 + 8192
    assert [int(wl.net.col[e]) for e in rep.path_edges[0]] == [1, 2]


def _ff_shortest(net, ff, s, d):
    dist = {s: 0}
    pq = [(0, s)]
    while pq:
        t, u = heapq.heappop(pq)
        if u == d:
            return t
        if t > dist.get(u, 1 << 62):
            continue
        for e in range(int(net.row_ptr[u]), int(net.row_ptr[u + 1])):
            v = int(net.col[e])
            if t + int(ff[e]) < dist.get(v, 1 << 62):
                dist[v] = t + int(ff[e])
                heapq.heappush(pq, (dist[v], v))
    return None


def test_fleet_invariants_city52(orc):
    wl = W.city52()
    src, dst = V.fleet(wl.net.n_nodes, 24, seed=5)
    rep = V.VehicleSim(OracleBackend(orc, wl), V.SimConfig(n_ants=16, n_iter=4, seed=3)).run(src, dst,
                                                                                            keep_paths=True)
    assert rep.arrived == 24
    ff = orc.prepare(orc.Net.from_workload(wl), orc.Params(), 0)["ff"]
    tails = wl.net.tails()
    taken = 0
    for i in range(24):
        p = rep.path_edges[i]
        taken += len(p)
        assert int(tails[p[0]]) == src[i] and int(wl.net.col[p[-1]]) == dst[i]
        assert all(int(wl.net.col[a]) == int(tails[b]) for a, b in zip(p, p[1:]))
        assert int(rep.trip_ms[i]) >= _ff_shortest(wl.net, ff, int(src[i]), int(dst[i]))
    assert rep.decisions == taken + rep.retries
    assert rep.makespan_s * 1000 == max(int(t) for t in rep.trip_ms)

"""Pins of the oracle's serving tick (queue / preemption update with dt > 0) against hand-worked
intersections, a millisecond simulation of the signal programme, and conservation of vehicles."""
import random

import numpy as np

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
from tests.test_oracle_primitives import _green_phase_at


def _junction(n02=5, n12=7):
    """0 -> 2 (phase 0) and 1 -> 2 (phase 1) feed node 2, which has out-roads 2 -> 3 and 2 -> 4.
    Roads are 100 m with 3 lanes (storage 40). Node 2: cycle 10 s, greens 4 s / 6 s, offset 0."""
    roads = [(0, 2, 1000, 50, 3, 0), (1, 2, 1000, 50, 3, 1), (2, 3, 1000, 50, 3, 0), (2, 4, 1000, 50, 3, 0)]
    net, sig, veh = NB.build(5, roads, signals={2: (10_000, 0, [4000, 6000])},
                             vehicles={(0, 2): n02, (1, 2): n12}, bidirectional=False)
    return net, sig, veh


def test_hand_worked_junction(orc):
    """t = 1 s lies in phase 0's window [0, 4 s): road 0->2 discharges min(5, 3 lanes * 2 s / 2 s) = 3;
    node 2 splits 3 over two out-roads as 2 (first in CSR order) and 1. Phase 1 keeps its 7 vehicles and
    its red time grows by dt. New queues (2, 7), storage 40 each (threshold 30), no red time above the
    cycle: the longest queue, phase 1, goes first."""
    net, sig, veh = _junction()
    onet = orc.Net(net, sig, veh)
    order = orc.queue_preempt(onet)
    assert list(order[2][:2]) == [1, 0]  # before the tick phase 1 already has the longer queue
    order[2][:2] = [0, 1]  # start from the default order so that phase 0 is green at t = 1 s
    v2, red, new_order = orc.tick(onet, orc.Params(), 1000, 2000, order)
    e = {(int(t), int(h)): i for i, (t, h) in enumerate(zip(net.tails(), net.col))}
    assert v2[e[(0, 2)]] == 2 and v2[e[(1, 2)]] == 7
    assert v2[e[(2, 3)]] == 2 and v2[e[(2, 4)]] == 1
    assert red[2][0] == 0 and red[2][1] == 2000
    assert list(new_order[2][:2]) == [1, 0]


def test_red_time_saturates(orc):
    """The red-time accumulator of a queued phase that is not green grows by dt and stops at 2^32 - 1
    instead of wrapping; the green phase's accumulator resets to 0."""
    net, sig, veh = _junction()
    red0 = np.zeros((5, 8), np.uint32)
    red0[2][:2] = [123, 2**32 - 1 - 500]
    onet = orc.Net(net, sig, veh, red0)
    order = orc.queue_preempt(onet)
    order[2][:2] = [0, 1]  # phase 0 green at t = 1 s
    _, red, _ = orc.tick(onet, orc.Params(), 1000, 2000, order)
    assert red[2][0] == 0 and red[2][1] == 2**32 - 1
    red0[2][1] = 2**32 - 1 - 2000  # exactly reaches the top
    _, red, _ = orc.tick(orc.Net(net, sig, veh, red0), orc.Params(), 1000, 2000, order)
    assert red[2][1] == 2**32 - 1


def test_green_phase_follows_the_programme(orc):
    """A star node with P phases, one loaded approach each: the approach that discharges is the one of
    the phase that a millisecond-by-millisecond simulation of the programme shows green."""
    rng = random.Random(4)
    for _ in range(200):
        P = rng.randint(1, 5)
        green = [rng.randint(1, 9) * 1000 for _ in range(P)]
        cycle = sum(green)
        offset = rng.randrange(cycle)
        roads = [(p, P, 1000, 50, 3, p) for p in range(P)] + [(P, P + 1, 1000, 50, 3, 0)]
        net, sig, veh = NB.build(P + 2, roads, signals={P: (cycle, offset, green)},
                                 vehicles={(p, P): 10 for p in range(P)}, bidirectional=False)
        sig.edge_phase[:] = net.orient
        onet = orc.Net(net, sig, veh)
        order = orc.queue_preempt(onet).copy()
        perm = list(range(P))
        rng.shuffle(perm)
        order[P][:P] = perm
        t_now = rng.randrange(0, 5 * cycle)
        v2, _, _ = orc.tick(onet, orc.Params(), t_now, 2000, order)
        tails = net.tails()
        served = [int(tails[i]) for i in range(net.n_edges) if net.col[i] == P and v2[i] < 10]
        assert served == [_green_phase_at(t_now, cycle, offset, green, perm)]


def test_conservation_on_grid(orc):
    """Every node of the grid has out-roads: the tick only moves vehicles."""
    wl = W.grid64(n_queries=1)
    onet = orc.Net.from_workload(wl)
    order = orc.queue_preempt(onet)
    veh = wl.vehicles.copy()
    red = np.zeros((wl.net.n_nodes, 8), np.uint32)
    moved = 0
    for k in range(5):
        v2, red, order = orc.tick(orc.Net(wl.net, wl.signals, veh, red), orc.Params(), 1000 * k, 1000, order)
        assert int(v2.sum()) == int(veh.sum())
        moved += int(np.abs(v2.astype(np.int64) - veh.astype(np.int64)).sum())
        veh = v2
    assert moved > 0


def test_sink_absorbs_and_unsignalised_node_serves_all(orc):
    """Node 2 is unsignalised: both approaches discharge. Node 3 has no out-road: what reaches it leaves."""
    roads = [(0, 2, 1000, 50, 3, 0), (1, 2, 1000, 50, 3, 1), (2, 3, 1000, 50, 3, 0)]
    net, sig, veh = NB.build(4, roads, vehicles={(0, 2): 4, (1, 2): 4, (2, 3): 5}, bidirectional=False)
    onet = orc.Net(net, sig, veh)
    v2, red, _ = orc.tick(onet, orc.Params(), 0, 2000, orc.queue_preempt(onet))
    e = {(int(t), int(h)): i for i, (t, h) in enumerate(zip(net.tails(), net.col))}
    assert v2[e[(0, 2)]] == 1 and v2[e[(1, 2)]] == 1  # 3 each served
    assert v2[e[(2, 3)]] == 5 - 3 + 6  # 3 discharged into the sink, 6 arrived from node 2
    assert int(v2.sum()) == int(veh.sum()) - 3
    assert int(red.sum()) == 0


def _two_phase(n0, n1, red1=0):
    """Approaches 0 -> 2 (phase 0) and 1 -> 2 (phase 1), 1 km and 3 lanes each (storage 400, threshold
    300); node 2 has cycle 20 s with greens 15 s / 5 s at offset 0 and one out-road."""
    roads = [(0, 2, 10000, 50, 3, 0), (1, 2, 10000, 50, 3, 1), (2, 3, 1000, 50, 3, 0)]
    net, sig, veh = NB.build(4, roads, signals={2: (20_000, 0, [15_000, 5_000])},
                             vehicles={(0, 2): n0, (1, 2): n1}, bidirectional=False)
    red = np.zeros((4, 8), np.uint32)
    red[2][1] = red1
    return net, sig, veh, red


def test_red_time_follows_the_programme(orc):
    """With the order held at (0, 1) (phase 0 keeps the longer queue, no queue over threshold, no red
    time over the cycle), phase 1 is green in [15 s, 20 s) of every cycle. After the tick at t (1 s
    steps from 0) phase 1's red time is (t mod 20 s) + 1 s inside [0, 15 s) and 0 inside its green;
    phase 0's is the mirror image."""
    net, sig, veh, red = _two_phase(250, 50)
    order = orc.queue_preempt(orc.Net(net, sig, veh))
    assert list(order[2][:2]) == [0, 1]
    for t in range(0, 60_000, 1000):
        veh, red, order = orc.tick(orc.Net(net, sig, veh, red), orc.Params(), t, 1000, order)
        c = t % 20_000
        assert red[2][1] == (c + 1000 if c < 15_000 else 0), t
        assert red[2][0] == (0 if c < 15_000 else c - 15_000 + 1000), t
        assert list(order[2][:2]) == [0, 1], t


def test_red_time_over_the_cycle_puts_the_phase_first(orc):
    """A red time that ends the tick above the cycle (20 s) puts phase 1 first; one that ends exactly
    at the cycle does not (the rule is strictly greater)."""
    for red1, first in ((19_500, 1), (19_000, 0)):
        net, sig, veh, red = _two_phase(250, 50, red1)
        order = orc.queue_preempt(orc.Net(net, sig, veh))
        _, red2, order2 = orc.tick(orc.Net(net, sig, veh, red), orc.Params(), 0, 1000, order)
        assert red2[2][1] == red1 + 1000
        assert order2[2][0] == first


def test_discharge_counts_the_whole_clock(orc):
    """3 lanes at h_sat = 2 s discharge 1.5 vehicles per second: 1-s ticks alternate 1, 2, 1, 2 ... so
    k ticks from t = 0 discharge exactly floor(1.5 k), as one tick of k seconds does."""
    roads = [(0, 1, 5000, 50, 3, 0), (1, 2, 1000, 50, 3, 0)]
    for k in (1, 2, 3, 7, 10):
        net, sig, veh = NB.build(3, roads, vehicles={(0, 1): 100}, bidirectional=False)
        red = np.zeros((3, 8), np.uint32)
        order = orc.queue_preempt(orc.Net(net, sig, veh))
        v = veh
        for t in range(k):
            v, red, order = orc.tick(orc.Net(net, sig, v, red), orc.Params(), 1000 * t, 1000, order)
        v1, _, _ = orc.tick(orc.Net(net, sig, veh), orc.Params(), 0, 1000 * k, order)
        e01 = next(i for i in range(net.n_edges) if net.col[i] == 1)
        assert v[e01] == 100 - (3 * k) // 2 == v1[e01]


def test_empty_phase_keeps_no_red_time(orc):
    """A phase whose approaches are empty accumulates no red time even while another phase is green."""
    net, sig, veh = _junction(n02=5, n12=0)
    red = np.zeros((5, 8), np.uint32)
    red[2][1] = 7000
    onet = orc.Net(net, sig, veh, red)
    order = orc.queue_preempt(onet)
    assert list(order[2][:2]) == [0, 1]
    _, red2, _ = orc.tick(onet, orc.Params(), 1000, 2000, order)
    assert red2[2][1] == 0 and red2[2][0] == 0

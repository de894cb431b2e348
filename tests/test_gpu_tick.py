"""Parity of the serving tick (gmp_tick) with the oracle's tick, bit for bit: vehicles on every road,
red-time accumulators, phase orders and road times after every tick of a long sequence; and a colony
solved on the ticked state equals the oracle's colony on the same state."""
import random

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


@pytest.fixture()
def ctx(gm):
    c = gm.Context(0)
    yield c
    c.close()


def _run_ticks(ctx, orc, net, sig, veh, n_ticks, seed, h_sat_ms=0, check_every=1):
    rng = random.Random(seed)
    prm = orc.Params(h_sat_ms=h_sat_ms)
    red = np.zeros((net.n_nodes, 8), np.uint32)
    order = orc.queue_preempt(orc.Net(net, sig, veh, red))
    t = rng.randrange(0, 100_000)
    for k in range(n_ticks):
        dt = rng.choice([0, 1, 250, 1000, 2000, 3700, 15_000])
        ctx.tick(t, dt)
        veh, red, order = orc.tick(orc.Net(net, sig, veh, red), prm, t, dt, order)
        t += dt
        if k % check_every == 0 or k == n_ticks - 1:
            np.testing.assert_array_equal(ctx.densities(), veh, err_msg=f"tick {k}")
            np.testing.assert_array_equal(ctx.red_times(), red, err_msg=f"tick {k}")
            np.testing.assert_array_equal(ctx.phase_order(), order, err_msg=f"tick {k}")
    prep = orc.prepare(orc.Net(net, sig, veh, red), prm, 0)
    tt, qd = ctx.edge_times()
    np.testing.assert_array_equal(tt, prep["tt"])
    np.testing.assert_array_equal(qd, prep["qd"])
    return veh, red, t


@pytest.mark.parametrize("name", ["grid10", "grid64"])
def test_tick_sequence_matches_oracle(gm, ctx, orc, name):
    wl = W.grid10() if name == "grid10" else W.grid64(n_queries=1)
    ctx.load_workload(wl)
    _run_ticks(ctx, orc, wl.net, wl.signals, wl.vehicles.copy(), 40, seed=11)


def test_tick_red_times_saturate(gm, ctx, orc):
    """Red-time accumulators a few seconds below 2^32 - 1 on every phase: the tick's growth saturates
    instead of wrapping, and the phase orders that follow (every queued phase starved, ties broken by
    phase index) match the oracle."""
    wl = W.grid10()
    rng = np.random.Generator(np.random.PCG64(31))
    red = (2**32 - 1 - rng.integers(0, 6000, size=(wl.net.n_nodes, 8))).astype(np.uint32)
    red[rng.random((wl.net.n_nodes, 8)) < 0.3] = 2**32 - 1
    ctx.load_workload(wl)
    ctx.set_red_times(red)
    onet = orc.Net(wl.net, wl.signals, wl.vehicles, red)
    order = orc.queue_preempt(onet)
    np.testing.assert_array_equal(ctx.phase_order(), order)
    veh = wl.vehicles.copy()
    t = 5000
    for dt in (3700, 1000, 0, 2000):
        ctx.tick(t, dt)
        veh, red, order = orc.tick(orc.Net(wl.net, wl.signals, veh, red), orc.Params(), t, dt, order)
        t += dt
        np.testing.assert_array_equal(ctx.densities(), veh)
        np.testing.assert_array_equal(ctx.red_times(), red)
        np.testing.assert_array_equal(ctx.phase_order(), order)
    assert (red == 2**32 - 1).sum() > 0


def test_tick_congested_and_custom_hsat(gm, ctx, orc):
    """Densities above the 3/4-storage threshold on many approaches (preemption by queue length) and
    a non-default saturation headway."""
    wl = W.grid64(n_queries=1)
    veh = (wl.vehicles.astype(np.uint64) * 12 + 7).astype(np.uint32)
    ctx.load_workload(wl)
    ctx.set_densities(veh)
    ctx.set_params(h_sat_ms=1700)
    _run_ticks(ctx, orc, wl.net, wl.signals, veh, 25, seed=12, h_sat_ms=1700)


def test_tick_sinks_and_unsignalised(gm, ctx, orc):
    """Nodes without out-roads absorb vehicles; unsignalised heads serve every approach."""
    rng = np.random.default_rng(5)
    roads = []
    for u in range(40):
        for v in rng.choice(60, size=rng.integers(1, 4), replace=False):
            if v != u:
                roads.append((u, int(v), int(rng.integers(300, 4000)), 50, int(rng.integers(1, 4)),
                              int(rng.integers(0, 2))))
    sigs = {v: (20_000, int(rng.integers(0, 20_000)), [12_000, 8_000]) for v in range(0, 60, 3)}
    net, sig, veh = NB.build(60, roads, signals=sigs, bidirectional=False)
    veh[:] = rng.integers(0, 60, size=veh.size)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    veh2, _, _ = _run_ticks(ctx, orc, net, sig, veh.copy(), 30, seed=13)
    assert int(veh2.sum()) < int(veh.sum())  # vehicles left through nodes 40..59's missing out-roads


def test_tick_high_in_degree_and_many_phases(gm, ctx, orc):
    """Intersections with up to 14 approaches (several rounds of four in the intersection passes) and 1 to
    6 phases (the two-phase rule and the general one), through a tick sequence: vehicles, red times,
    phase orders and road records after every tick equal the oracle's."""
    rng = np.random.default_rng(21)
    n = 80
    hubs = list(range(0, n, 10))
    roads = {}
    for h in hubs:
        for u in rng.choice([x for x in range(n) if x != h], size=int(rng.integers(6, 15)), replace=False):
            roads[(int(u), h)] = (int(rng.integers(300, 4000)), 50, int(rng.integers(1, 4)), int(rng.integers(0, 2)))
    for u in range(n):
        for v in rng.choice(n, size=2, replace=False):
            if int(v) != u and (u, int(v)) not in roads:
                roads[(u, int(v))] = (int(rng.integers(300, 4000)), 60, int(rng.integers(1, 4)), int(rng.integers(0, 2)))
    sigs = {}
    for k, h in enumerate(hubs):
        g = [int(x) for x in rng.integers(5000, 20000, [1, 2, 2, 3, 4, 5, 6, 2][k])]
        sigs[h] = (sum(g), int(rng.integers(0, sum(g))), g)
    for v in range(1, n, 3):
        sigs.setdefault(v, (20_000, int(rng.integers(0, 20_000)), [12_000, 8_000]))
    net, sig, veh = NB.build(n, [(a, b, *r) for (a, b), r in sorted(roads.items())], signals=sigs,
                             bidirectional=False)
    ep = sig.edge_phase.copy()
    for e in range(net.n_edges):  # approaches spread over every phase of their head
        P = int(sig.n_phases[net.col[e]])
        ep[e] = rng.integers(0, P) if P > 2 else (0 if P == 1 else ep[e])
    sig = W.SignalTiming(sig.n_phases, sig.cycle_ms, sig.offset_ms, sig.green_ms, ep)
    assert np.bincount(net.col, minlength=n).max() > 8
    veh[:] = rng.integers(0, 60, size=veh.size)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    _run_ticks(ctx, orc, net, sig, veh.copy(), 30, seed=15)


def test_solve_after_ticks_matches_oracle(gm, ctx, orc):
    wl = W.grid10()
    ctx.load_workload(wl)
    veh, red, t = _run_ticks(ctx, orc, wl.net, wl.signals, wl.vehicles.copy(), 12, seed=14, check_every=4)
    onet = orc.Net(wl.net, wl.signals, veh, red)
    t_dep = t % (1 << 29)
    ctx.set_params(t_dep_ms=t_dep)
    q = W.Query(3, 96, 32, 6, 1.0, 2.0, 0.1, 99)
    g = ctx.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed)
    o = orc.solve(onet, orc.Params(t_dep_ms=t_dep), q)
    assert g["status"] == o["status"] == 0
    assert g["travel_ms"] == o["travel_ms"] and g["wait_ms"] == o["wait_ms"]
    np.testing.assert_array_equal(g["route"], o["route"])


def test_tick_argument_errors(gm, ctx):
    with pytest.raises(gm.GmpError) as ei:
        ctx.tick(0, 1000)
    assert ei.value.code == gm.ERR_STATE
    ctx.load_workload(W.grid10())
    with pytest.raises(gm.GmpError) as ei:
        ctx.tick((1 << 48) + 1, 1000)
    assert ei.value.code == gm.ERR_INVALID_ARG
    with pytest.raises(gm.GmpError) as ei:
        ctx.tick(0, (1 << 30) + 1)
    assert ei.value.code == gm.ERR_INVALID_ARG

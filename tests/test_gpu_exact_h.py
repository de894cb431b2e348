"""Parity of the exact Calc_Dist option (GMP_FLAG_EXACT_H: the GPU's per-colony shortest-time relaxation
from the destination) with the oracle's Dijkstra, through whole colonies: routes, times, step and success
counts, per-ant logs and final pheromone tables are equal bit for bit, so every colony's heuristic table
and deposit numerator are too. Covered: every schedule, one-way graphs where some nodes cannot reach the
destination (the clamp), congested and ticked traffic, and the 100k-node graph."""
import dataclasses
import multiprocessing as mp

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
from tests.test_gpu_parity import SCHEDULES, _compare, _with_flags

pytestmark = pytest.mark.gpu

Q = W.Query
EXACT = 256


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


@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_grid10_exact_h(gm, ctx, orc, sched):
    wl = W.grid10(n_ants=32, n_iter=12)
    ctx.load_workload(wl)
    ctx.set_params(**_with_flags(sched, EXACT | gm.FLAG_ANT_LOG))
    q = wl.queries[0]
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(flags=EXACT), q, r, ctx, 0, ctx.ant_log(0))


@pytest.mark.parametrize("sched", ["chains_default", "persistent", "sparse_tau"])
def test_grid64_exact_h_batch(gm, ctx, orc, sched):
    wl = W.grid64(n_queries=4, n_ants=256, n_iter=12)
    ctx.load_workload(wl)
    ctx.set_params(**_with_flags(sched, EXACT | gm.FLAG_ANT_LOG))
    res = ctx.solve_batch(wl.queries)
    onet = orc.Net.from_workload(wl)
    for i, q in enumerate(wl.queries):
        _compare(orc, onet, orc.Params(flags=EXACT), q, res[i], ctx, i, ctx.ant_log(i))


def test_one_way_graph_with_unreachable_nodes(gm, ctx, orc):
    """Random one-way roads: some sources cannot reach their destination (h = 2^28 everywhere on the way)."""
    rng = np.random.default_rng(17)
    n = 80
    a = rng.integers(0, n, 260)
    b = (a + rng.integers(1, n, 260)) % n
    roads = [(int(x), int(y), int(rng.integers(1000, 5000)), int(rng.choice([30, 50, 70]))) for x, y in zip(a, b)]
    net, sig, veh = NB.build(n, roads, [(int(rng.integers(0, 9000)), int(rng.integers(0, 9000))) for _ in range(n)],
                             bidirectional=False)
    veh = rng.integers(0, 50, net.n_edges).astype(np.uint32)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    ctx.set_params(flags=EXACT)
    qs = [Q(int(s), int(d), 24, 6, 1.0, 2.0, 0.1, 40 + i) for i, (s, d) in enumerate(W.uniform_od(n, 12, rng))]
    res = ctx.solve_batch(qs)
    onet = orc.Net(net, sig, veh)
    statuses = set()
    for i, q in enumerate(qs):
        o = _compare(orc, onet, orc.Params(flags=EXACT), q, res[i], ctx, i)
        statuses.add(o["status"])
        assert int(orc.prepare(onet, orc.Params(flags=EXACT), q.dst)["h"].max()) <= 2**28
    assert (orc.prepare(onet, orc.Params(flags=EXACT), qs[0].dst)["h"] == 2**28).any()


def test_exact_h_after_ticks(gm, ctx, orc):
    """The bound follows the traffic: after serving ticks move vehicles, the colony (and its bound) uses
    the new travel times."""
    wl = W.grid10(n_ants=24, n_iter=6)
    ctx.load_workload(wl)
    veh, red = wl.vehicles.copy(), np.zeros((wl.net.n_nodes, 8), np.uint32)
    order = orc.queue_preempt(orc.Net(wl.net, wl.signals, veh, red))
    for t, dt in [(0, 3000), (3000, 2000)]:
        ctx.tick(t, dt)
        veh, red, order = orc.tick(orc.Net(wl.net, wl.signals, veh, red), orc.Params(), t, dt, order)
    ctx.set_params(flags=EXACT, t_dep_ms=5000)
    q = dataclasses.replace(wl.queries[0], seed=9)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net(wl.net, wl.signals, veh, red), orc.Params(flags=EXACT, t_dep_ms=5000), q, r, ctx)


def _oracle_geo(qi):
    from oracle import oracle as orc

    wl = W.geo100k(n_queries=64)
    q = dataclasses.replace(wl.queries[qi], n_ants=64, n_iter=10)
    return orc.solve(orc.Net.from_workload(wl), orc.Params(flags=EXACT), q, want_tau=False)


def test_geo100k_exact_h_sampled(gm):
    """64 colonies of the 100k-node graph (visited sets in global memory); two re-solved by the oracle."""
    sample = (0, 63)
    pool = mp.get_context("spawn").Pool(len(sample))
    pending = pool.map_async(_oracle_geo, sample)
    wl = W.geo100k(n_queries=64)
    qs = [dataclasses.replace(q, n_ants=64, n_iter=10) for q in wl.queries]
    ctx = gm.Context(0)
    try:
        ctx.load_workload(wl)
        ctx.set_params(flags=EXACT)
        res = ctx.solve_batch(qs)
    finally:
        ctx.close()
    oracle = pending.get(timeout=1800)
    pool.close()
    for qi, o in zip(sample, oracle):
        r = res[qi]
        assert r["status"] == o["status"]
        for k in ("travel_ms", "wait_ms", "ant_steps", "n_success", "best_iter", "best_ant"):
            assert r[k] == o[k], (qi, k, r[k], o[k])

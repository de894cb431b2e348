"""Many road graphs in one launch: every colony of every graph equals its graph's batch launched alone,
and a sample equals the oracle bit for bit; at full size (64 city graphs), every colony of one graph per
size bucket equals the oracle."""
import dataclasses

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import oracle_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


def _same(a, b):
    for k in ("status", "travel_ms", "wait_ms", "ant_steps", "n_success", "best_iter", "best_ant", "route_len"):
        assert a[k] == b[k], (k, a[k], b[k])
    np.testing.assert_array_equal(a["route"], b["route"])


def test_city_batch_one_launch(gm, orc):
    cities = W.city_batch(n_graphs=6, n_min=500, n_max=20_000, q_lo=2, q_hi=5, ants_lo=32, ants_hi=160, n_iter=6)
    cities.append(W.grid10())
    ctxs = []
    m = gm.Multi(0)
    try:
        for wl in cities:
            c = gm.Context(0)
            c.load_workload(wl)
            ctxs.append(c)
        batches = [wl.queries for wl in cities]
        res = m.solve(ctxs, batches)
        res2 = m.solve(ctxs, batches)  # replayed capture, fresh pheromone: identical
        for r1, r2 in zip(res, res2):
            for a, b in zip(r1, r2):
                _same(a, b)
        # a changed batch on one graph is re-captured
        batches[0] = [dataclasses.replace(q, seed=q.seed + 1) for q in batches[0]][:1]
        res3 = m.solve(ctxs, batches)
        assert len(res3[0]) == 1
        for c, wl, qs, r in zip(ctxs, cities, batches, res3):
            alone = c.solve_batch(qs)
            for a, b in zip(r, alone):
                _same(a, b)
        for gi in (1, len(cities) - 1):  # oracle on a sample of graphs
            onet = orc.Net.from_workload(cities[gi])
            for q, r in zip(batches[gi], res3[gi]):
                o = orc.solve(onet, orc.Params(), q, want_tau=False)
                assert r["status"] == o["status"] and r["travel_ms"] == o["travel_ms"]
                assert r["ant_steps"] == o["ant_steps"]
                if o["status"] == 0:
                    np.testing.assert_array_equal(r["route"], o["route"])
    finally:
        m.close()
        for c in ctxs:
            c.close()


def test_city_batch_full_size(gm):
    """The 64-graph workload (1.1k-187k nodes, 2362 colonies of 128-1024 ants, 50 iterations) in one
    launch. In each size bucket of node counts (1k-4k, 4k-16k, 16k-64k, 64k-200k) the first graph has
    every colony re-solved by the oracle, and each must agree bit for bit, final pheromone table included.
    Every route of every graph is valid."""
    cities = W.city_batch()
    ns = [wl.net.n_nodes for wl in cities]
    edges = [1000, 4000, 16000, 64000, 200001]
    pick = [next(g for g in range(len(cities)) if lo <= ns[g] < hi) for lo, hi in zip(edges[:-1], edges[1:])]
    items = [(g, qi) for g in pick for qi in range(len(cities[g].queries))]
    pool, pending = oracle_pool.start("city_batch", items)
    ctxs = []
    m = gm.Multi(0)
    try:
        for wl in cities:
            c = gm.Context(0)
            c.load_workload(wl)
            ctxs.append(c)
        res = m.solve(ctxs, [wl.queries for wl in cities])
        digests = {(g, qi): oracle_pool.tau_digest(ctxs[g].pheromone(qi)) for g, qi in items}
        for wl, rs in zip(cities, res):
            assert len(rs) == len(wl.queries)
            for q, r in zip(wl.queries, rs):
                assert r["ant_steps"] > 0 and r["status"] in (0, gm.ERR_NO_ROUTE)
                if r["status"] != 0:
                    continue
                route = r["route"]
                assert route[0] == q.src and route[-1] == q.dst and len(set(route.tolist())) == len(route)
                for a, b in zip(route[:-1], route[1:]):
                    assert b in wl.net.col[wl.net.row_ptr[a]:wl.net.row_ptr[a + 1]]
        oracle = pending.get(timeout=3000)
    finally:
        pool.close()
        pool.join()
        m.close()
        for c in ctxs:
            c.close()
    assert [it for it, _ in oracle] == items
    for (g, qi), o in oracle:
        oracle_pool.check(res[g][qi], o)
        assert digests[(g, qi)] == o["tau_sha256"], (g, qi)


def test_multi_refuses(gm):
    m = gm.Multi(0)
    c = gm.Context(0)
    try:
        c.load_workload(W.grid10())
        with pytest.raises(gm.GmpError) as ei:
            m.launch([c])
        assert ei.value.code == gm.ERR_STATE
        c.stage(W.grid10().queries)
        with pytest.raises(gm.GmpError) as ei:
            m.launch([c, c])
        assert ei.value.code == gm.ERR_INVALID_ARG
        c.set_params(mode=gm.MODE_PERSISTENT)
        c.stage(W.grid10().queries)
        with pytest.raises(gm.GmpError) as ei:
            m.launch([c])
        assert ei.value.code == gm.ERR_UNSUPPORTED
    finally:
        m.close()
        c.close()


def test_graphs_with_different_shared_memory_sizes(gm, orc):
    """Two graphs whose visited bitmaps need different amounts of shared memory above the default
    48 KB (30k and 26k nodes: 60 KB and 52 KB per block at 8 lanes per ant), staged one after the other
    and launched together."""
    rng = np.random.Generator(np.random.PCG64(21))
    wls = []
    for rows in (150, 130):
        net = W.geometric_network(rows, 200, rng)
        sig = W.two_phase_signals(net, rng.random(net.n_nodes) < 0.6, rng)
        veh = W.vehicles_poisson(net.n_edges, 1.0, rng)
        od = W.uniform_od(net.n_nodes, 2, rng)
        qs = [W.Query(s, d, 32, 3, 1.0, 2.0, 0.1, 50 + i) for i, (s, d) in enumerate(od)]
        wls.append(W.Workload(f"geo{rows}", net, sig, veh, qs))
    m = gm.Multi(0)
    ctxs = []
    try:
        for wl in wls:
            c = gm.Context(0)
            c.load_workload(wl)
            c.set_params(lanes_per_ant=8, mode=1)
            ctxs.append(c)
        res = m.solve(ctxs, [wl.queries for wl in wls])
        for wl, rr in zip(wls, res):
            onet = orc.Net.from_workload(wl)
            for q, r in zip(wl.queries, rr):
                o = orc.solve(onet, orc.Params(), q, want_tau=False)
                assert r["status"] == o["status"] and r["travel_ms"] == o["travel_ms"]
                assert r["ant_steps"] == o["ant_steps"]
    finally:
        m.close()
        for c in ctxs:
            c.close()


def test_variants_in_one_launch(gm, orc):
    """Graphs whose contexts use different options share one launch: the exact heuristic with the
    paper-literal pheromone rules, non-integer exponents, and the defaults. Each equals its graph alone
    and the oracle."""
    cities = W.city_batch(n_graphs=3, n_min=500, n_max=3000, q_lo=2, q_hi=3, ants_lo=32, ants_hi=64, n_iter=5)
    opts = [dict(flags=gm.FLAG_EXACT_H | gm.FLAG_PAPER_LITERAL), dict(), dict(flags=gm.FLAG_EXACT_H)]
    batches = [wl.queries for wl in cities]
    batches[1] = [dataclasses.replace(q, alpha=1.5, beta=2.25) for q in batches[1]]
    ctxs = []
    m = gm.Multi(0)
    try:
        for wl, o in zip(cities, opts):
            c = gm.Context(0)
            c.load_workload(wl)
            c.set_params(**o)
            ctxs.append(c)
        res = m.solve(ctxs, batches)
        for c, qs, r in zip(ctxs, batches, res):
            for a, b in zip(r, c.solve_batch(qs)):
                _same(a, b)
        for wl, o, qs, r in zip(cities, opts, batches, res):
            onet = orc.Net.from_workload(wl)
            q, got = qs[0], r[0]
            exp = orc.solve(onet, orc.Params(flags=o.get("flags", 0)), q, want_tau=False)
            for k in ("status", "travel_ms", "ant_steps", "n_success"):
                assert got[k] == exp[k], (k, got[k], exp[k])
    finally:
        m.close()
        for c in ctxs:
            c.close()

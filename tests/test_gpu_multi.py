"""Many road graphs in one launch: every colony of every graph equals its graph's batch launched alone,
and a sample equals the oracle bit for bit."""
import dataclasses

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W

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

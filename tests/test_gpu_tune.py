"""The autotuner changes speed only: after tuning, a batch still equals the oracle bit for bit; the
second call in the same size bucket reuses the cached choice; and every queue chunk of the persistent
job gives the same results."""
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


@pytest.fixture()
def ctx(gm):
    c = gm.Context(0)
    yield c
    c.close()


def _check_batch(orc, wl, res, queries):
    onet = orc.Net.from_workload(wl)
    for q, g in zip(queries, res):
        o = orc.solve(onet, orc.Params(), q, want_tau=False)
        assert g["status"] == o["status"]
        assert g["travel_ms"] == o["travel_ms"] and g["wait_ms"] == o["wait_ms"]
        assert g["ant_steps"] == o["ant_steps"] and g["n_success"] == o["n_success"]
        if o["status"] == 0:
            np.testing.assert_array_equal(g["route"], o["route"])


@pytest.mark.parametrize("name", ["grid10", "grid64"])
def test_autotune_then_parity_and_cache(gm, orc, name):
    gm.Context.autotune_reset()
    wl = W.grid10() if name == "grid10" else W.grid64(n_queries=4)
    queries = [dataclasses.replace(q, n_ants=96, n_iter=5, seed=q.seed + 7) for q in wl.queries]
    c1 = gm.Context(0)
    try:
        c1.load_workload(wl)
        t = c1.autotune(queries, probe_iter=3)
        assert t["from_cache"] == 0 and t["n_tried"] >= 6
        assert 0 < t["best_ms"] <= t["default_ms"]
        assert t["lanes_per_ant"] in (1, 4, 8, 16, 32) and t["mode"] in (1, 2)
        p = c1.get_params()
        assert p["lanes_per_ant"] == t["lanes_per_ant"] and p["mode"] == t["mode"]
        _check_batch(orc, wl, c1.solve_batch(queries), queries)
    finally:
        c1.close()
    c2 = gm.Context(0)
    try:
        c2.load_workload(wl)
        t2 = c2.autotune(queries, probe_iter=3)
        assert t2["from_cache"] == 1 and t2["n_tried"] == 0 and t2["bucket"] == t["bucket"]
        assert (t2["lanes_per_ant"], t2["mode"], t2["queue_chunk"]) == (t["lanes_per_ant"], t["mode"],
                                                                        t["queue_chunk"])
        _check_batch(orc, wl, c2.solve_batch(queries), queries)
    finally:
        c2.close()


@pytest.mark.parametrize("chunk", [8, 32, 64])
def test_persistent_queue_chunk_parity(gm, ctx, orc, chunk):
    wl = W.grid10()
    queries = [dataclasses.replace(wl.queries[0], n_ants=40, n_iter=6, seed=s) for s in (1, 2, 3)]
    ctx.load_workload(wl)
    ctx.set_params(mode=gm.MODE_PERSISTENT, lanes_per_ant=8, queue_chunk=chunk)
    _check_batch(orc, wl, ctx.solve_batch(queries), queries)
    np.testing.assert_array_equal(ctx.phase_order(), orc.prepare(orc.Net.from_workload(wl), orc.Params(), 0)["order"])


def test_queue_chunk_rejects_other_values(gm, ctx):
    ctx.load_workload(W.grid10())
    with pytest.raises(gm.GmpError) as ei:
        ctx.set_params(queue_chunk=12)
    assert ei.value.code == gm.ERR_INVALID_ARG

"""The 100k-node planar graph at full size: 512 colonies x 256 ants x 100 iterations in one job (visited
sets in global memory, 16 concurrent chains). Three colonies spread over the chains are re-solved by the
oracle and must agree bit for bit; every route found is checked for validity. (On this sparse planar
graph with 20-400 hop pairs most ants end in dead ends under the simple-path rule, so few or no colonies
find a route; the counts of steps and successes still pin the whole walk.)"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SAMPLE = (0, 255, 511)


def _oracle_one(qi):
    from oracle import oracle as orc

    wl = W.geo100k()
    return orc.solve(orc.Net.from_workload(wl), orc.Params(), wl.queries[qi], want_tau=False)


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


def test_geo100k_full_size_sampled(gm):
    # the oracle processes start before the first GPU call (spawn: no CUDA state is inherited)
    pool = mp.get_context("spawn").Pool(len(SAMPLE))
    pending = pool.map_async(_oracle_one, SAMPLE)
    wl = W.geo100k()
    ctx = gm.Context(0)
    try:
        ctx.load_workload(wl)
        res = ctx.solve_batch(wl.queries)
    finally:
        ctx.close()
    net = wl.net
    for q, r in zip(wl.queries, res):
        assert r["ant_steps"] > 0 and r["status"] in (0, gm.ERR_NO_ROUTE)
        if r["status"] != 0:
            continue
        route = r["route"]
        assert route[0] == q.src and route[-1] == q.dst and len(set(route.tolist())) == len(route)
        for a, b in zip(route[:-1], route[1:]):
            row = net.col[net.row_ptr[a]:net.row_ptr[a + 1]]
            assert b in row
    oracle = pending.get(timeout=1800)
    pool.close()
    for qi, o in zip(SAMPLE, oracle):
        r = res[qi]
        assert r["status"] == o["status"]
        for k in ("travel_ms", "wait_ms", "ant_steps", "n_success"):
            assert r[k] == o[k], (qi, k, r[k], o[k])
        if o["status"] == 0:
            assert r["best_iter"] == o["best_iter"] and r["best_ant"] == o["best_ant"]
            np.testing.assert_array_equal(r["route"], o["route"])

"""The 100k-node planar graph at full size: 512 colonies x 256 ants x 100 iterations in one job (visited
sets in global memory, 16 concurrent chains, sparse pheromone). Every colony is re-solved by the oracle
(a pool of spawned processes over the host cores) and must agree bit for bit: status, best route, travel
and wait times, ant-step and success counts, best (iteration, ant) and the final pheromone table (by
digest). Every route found is also checked for validity, and at least 90 % of the colonies must find
one: ants step back out of dead ends, so on this sparse planar graph (20-400 hop pairs, 8 % of nodes
with one road out) nearly every ant reaches its destination."""
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


N_COLONIES = 512


def test_geo100k_full_size_full_parity(gm):
    # the workers build the workload while this process builds its own and runs the job
    pool, pending = oracle_pool.start("geo100k", range(N_COLONIES))
    try:
        wl = W.geo100k()
        assert len(wl.queries) == N_COLONIES
        ctx = gm.Context(0)
        try:
            ctx.load_workload(wl)
            res = ctx.solve_batch(wl.queries)
            digests = [oracle_pool.tau_digest(ctx.pheromone(i)) for i in range(len(wl.queries))]
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
        oracle = pending.get(timeout=3000)
    finally:
        pool.close()
        pool.join()
    assert [qi for qi, _ in oracle] == list(range(N_COLONIES))
    for qi, o in oracle:
        oracle_pool.check(res[qi], o)
        assert digests[qi] == o["tau_sha256"], qi
    routed = sum(r["status"] == 0 for r in res)
    assert routed >= 0.9 * N_COLONIES, routed
    assert sum(r["n_success"] for r in res) >= 0.5 * sum(q.n_ants * q.n_iter for q in wl.queries)

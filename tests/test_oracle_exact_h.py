"""Pins of the oracle's exact Calc_Dist (the least congested travel time from each node to the destination):
scipy's Dijkstra on the reversed graph, brute force over simple paths on tiny graphs, the clamp for nodes
that cannot reach the destination, admissibility against the colony's best routes, and the deposit
numerator that follows from it. No GPU needed."""
import itertools

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB

Q = W.Query
CLAMP = 2 ** 28


def _scipy_h(net, tt, dst):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra

    tails = net.tails()
    # duplicate (tail, head) roads: keep the faster one, as a path would
    best = {}
    for e in range(net.n_edges):
        k = (int(net.col[e]), int(tails[e]))
        best[k] = min(best.get(k, 1 << 62), int(tt[e]))
    r = np.array([k[0] for k in best]), np.array([k[1] for k in best])
    w = np.array(list(best.values()), float)
    w[w == 0] = 1e-9  # a zero-weight entry would vanish from the sparse matrix
    M = csr_matrix((w, r), shape=(net.n_nodes, net.n_nodes))
    d = dijkstra(M, indices=dst)
    return np.where(np.isinf(d), CLAMP, np.minimum(np.round(d), CLAMP)).astype(np.int64)


@pytest.mark.parametrize("case", ["grid10", "grid64", "random", "directed"])
def test_exact_h_equals_scipy_dijkstra(orc, case):
    rng = np.random.default_rng(4)
    if case == "grid10":
        wl = W.grid10()
        net, sig, veh = wl.net, wl.signals, wl.vehicles
    elif case == "grid64":
        wl = W.grid64(n_queries=1)
        net, sig, veh = wl.net, wl.signals, wl.vehicles
    elif case == "random":
        net, sig = W.random_small(300, 700, rng, signalised_frac=0.5)
        veh = rng.integers(0, 40, net.n_edges).astype(np.uint32)
    else:  # one-way roads: some nodes cannot reach the destination
        n = 60
        a = rng.integers(0, n, 150)
        b = (a + rng.integers(1, n, 150)) % n
        roads = [(int(x), int(y), int(rng.integers(1000, 5000)), 50) for x, y in zip(a, b)]
        net, sig, veh = NB.build(n, roads, bidirectional=False)
    onet = orc.Net(net, sig, veh)
    for dst in rng.choice(net.n_nodes, 4, replace=False):
        p = orc.prepare(onet, orc.Params(flags=orc.FLAG_EXACT_H), int(dst))
        np.testing.assert_array_equal(p["h"].astype(np.int64), _scipy_h(net, p["tt"], int(dst)))
        assert p["h"][dst] == 0
    if case == "directed":
        assert (p["h"] == CLAMP).any()


def test_exact_h_brute_force_tiny(orc):
    rng = np.random.default_rng(9)
    for g in range(20):
        net, sig = W.random_small(7, 10, rng, signalised_frac=0.0)
        veh = rng.integers(0, 30, net.n_edges).astype(np.uint32)
        onet = orc.Net(net, sig, veh)
        dst = int(rng.integers(0, 7))
        p = orc.prepare(onet, orc.Params(flags=orc.FLAG_EXACT_H), dst)
        tails = net.tails()
        for v in range(7):
            best = CLAMP if v != dst else 0
            # every simple path v -> dst: sequences of distinct intermediate nodes
            others = [u for u in range(7) if u not in (v, dst)]
            for k in range(len(others) + 1):
                for mid in itertools.permutations(others, k):
                    nodes = [v, *mid, dst]
                    tot = 0
                    for x, y in zip(nodes, nodes[1:]):
                        es = [e for e in range(net.n_edges) if tails[e] == x and net.col[e] == y]
                        if not es:
                            break
                        tot += min(int(p["tt"][e]) for e in es)
                    else:
                        if v != dst:
                            best = min(best, tot)
            assert int(p["h"][v]) == best, (g, v)


def test_exact_h_is_admissible_and_sharper(orc):
    """Every node's exact bound is at least its straight-line bound, and no colony finds a route from the
    source faster than the bound (waits only add to the travel times it sums)."""
    wl = W.grid64(n_queries=3, n_ants=64, n_iter=8)
    onet = orc.Net.from_workload(wl)
    for q in wl.queries:
        pe = orc.prepare(onet, orc.Params(flags=orc.FLAG_EXACT_H), q.dst)
        pg = orc.prepare(onet, orc.Params(), q.dst)
        assert (pe["h"] >= pg["h"]).all()
        for flags in (0, orc.FLAG_EXACT_H):
            r = orc.solve(onet, orc.Params(flags=flags), q, want_tau=False)
            if r["status"] == 0:
                assert r["travel_ms"] >= int(pe["h"][q.src])


def test_exact_h_deposit_numerator(orc):
    """One iteration: sum of tau' = E * evap(1.0) + sum over successful ants of |route| * floor(h(src) * 2^32 / T)
    with the exact h(src)."""
    wl = W.grid10(n_ants=32, n_iter=1)
    onet = orc.Net.from_workload(wl)
    q = wl.queries[0]
    prm = orc.Params(flags=orc.FLAG_EXACT_H)
    h_src = int(orc.prepare(onet, prm, q.dst)["h"][q.src])
    r = orc.solve(onet, prm, q, want_log=True)
    st, length, _, T, _ = orc.log_fields(r["log"][0])
    dep = sum(int(n) * ((max(h_src, 1) << 32) // int(t)) for n, t in zip(length[st == 0], T[st == 0]))
    assert dep > 0
    assert int(r["tau"].sum()) == wl.net.n_edges * orc.evaporate(2 ** 32, orc.rho_fix(q.rho)) + dep

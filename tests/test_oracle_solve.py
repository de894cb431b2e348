"""Pins of the oracle's ant walk and full colony against hand-worked steps, textbook shortest-path
routines, brute force, exact identities and degenerate cases. No GPU needed."""
import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
from tests.test_oracle_primitives import _exact_weights

Q = W.Query


def _star(signal_on_1=False, veh01=0, far1=False):
    """Node 0 -> {1, 2, 3} -> 4. Roads at 45 km/h; lengths 512 / 1024 / 256 dm give free-flow
    times of exactly 4096 / 8192 / 2048 ms."""
    roads = [(0, 1, 512, 45, 3, 0), (0, 2, 1024, 45, 3, 0), (0, 3, 256, 45, 3, 0),
             (1, 4, 512, 45, 3, 1), (2, 4, 512, 45, 3, 0), (3, 4, 512, 45, 3, 0)]
    coords = [(0, 0)] * 5
    if far1:
        coords[1] = (3000, 4000)  # 500 m from the destination; 8 ms/dm at 45 km/h -> h = 40000 ms
    signals = {1: (10_000, 0, [4000, 6000])} if signal_on_1 else None
    vehicles = {(0, 1): veh01} if veh01 else None
    return NB.build(5, roads, coords, signals, vehicles)


def test_hand_worked_first_step_kat_draw(orc):
    """Three candidates with scores 2^-12, 2^-13, 2^-11 (alpha=beta=1, tau=1.0, h=0, no signals):
    weights 2^21, 2^20, 2^22; S = 7*2^20. The draw for (seed 0, it 0, ant 0, step 0) is the first
    Philox known-answer vector, 0xe169c58d6627e8d5 / 2^64 = 0.8805..., so r = 6.16 * 2^20 lies in
    [3*2^20, 7*2^20): the third road (0 -> 3). Then 3 -> 4 is the only choice: T = 2048 + 4096."""
    net, sig, veh = _star()
    onet = orc.Net(net, sig, veh)
    tau = np.full(net.n_edges, 2**32, np.uint64)
    w = orc.walk_one(onet, orc.Params(), Q(0, 4, 1, 1, 1.0, 1.0, 0.1, 0), tau, it=0, ant=0)
    assert w["status"] == 0
    assert [int(net.col[e]) for e in w["route_edges"]] == [3, 4]
    assert w["T"] == 6144 and w["W"] == 0 and w["steps"] == 2


def _expected_pick(orc, weights, seed, it, ant, step):
    o = orc.philox([it, ant, step, 0], [seed & 0xFFFFFFFF, seed >> 32])
    rnd = o[0] | (o[1] << 32)
    r = (rnd * sum(weights)) >> 64
    acc = 0
    for i, w in enumerate(weights):
        acc += w
        if acc > r:
            return i


def test_hand_worked_step_with_signal_queue_and_heuristic(orc):
    """Road 0->1 carries 3 vehicles: cap = 3*512/75 = 20, tt = 4096*20/17 = 4818 ms. Node 1 is
    signalised (cycle 10 s, phase 0 green [0, 4 s) from offset 0; phase order stays [0, 1] since
    Q_0 = 3 is the longest queue); arrival at 4818 ms waits 10000 - 4818 = 5182 ms, plus queue delay
    3*2000/3 = 2000 ms. Node 1 lies 500 m from the destination: h = 5000 dm * 8 ms/dm = 40000 ms.
    So c = 4818 + 7182 + 40000 = 52000 for road 0->1, 8192 for 0->2, 2048 for 0->3."""
    net, sig, veh = _star(signal_on_1=True, veh01=3, far1=True)
    onet = orc.Net(net, sig, veh)
    prep = orc.prepare(onet, orc.Params(), 4)
    e01 = NB.edge_id(net, 0, 1)
    assert prep["tt"][e01] == 4818 and prep["qd"][e01] == 2000 and prep["h"][1] == 40000
    f32 = np.float32
    scores = [f32(1) / f32(52000), f32(1) / f32(8192), f32(1) / f32(2048)]
    weights = _exact_weights(scores)
    tau = np.full(net.n_edges, 2**32, np.uint64)
    heads = []
    for ant in range(300):
        w = orc.walk_one(onet, orc.Params(), Q(0, 4, 300, 1, 1.0, 1.0, 0.1, 77), tau, it=0, ant=ant)
        pick = _expected_pick(orc, weights, 77, 0, ant, 0)
        assert int(net.col[w["route_edges"][0]]) == [1, 2, 3][pick]
        heads.append(pick)
        if pick == 0:  # went through the signal: T = 52000 - 40000 + road 1->4 (4096 ms)
            assert w["T"] == 4818 + 7182 + 4096 and w["W"] == 7182
    assert set(heads) == {0, 1, 2}


def _line_net(orc, xs, roads, dst_first=False):
    """Nodes on the x axis at xs (dm); roads (a, b, length_dm) both ways at 45 km/h, the fastest road, so
    the straight-line bound is exactly 8 ms per dm and a road of L dm takes exactly 8*L ms."""
    net, sig, veh = NB.build(len(xs), [(a, b, L, 45) for a, b, L in roads], [(x, 0) for x in xs])
    return net, orc.Net(net, sig, veh)


def test_hand_worked_step_reduced_cost(orc):
    """Q2's reading: a road costs the time it adds over the remaining bound, c = tt + wait + h(v) - h(u).
    src 0 at x = 512, node 1 at 768, node 2 at 0, destination 3 at 1536; roads 0-1 and 0-2 of 512 dm
    (4096 ms). h(0) = 1024*8 = 8192, h(1) = 6144, h(2) = 12288, so c(0->1) = 4096 + 6144 - 8192 = 2048
    and c(0->2) = 4096 + 12288 - 8192 = 8192: scores 2^-11 and 2^-13, weights 2^22 and 2^20, chances
    4/5 and 1/5 (without the -h(u) term they would be 10240 and 16384). Via 1 the ant takes road 1-3
    (768 dm, 6144 ms), via 2 road 2-3 (1536 dm, 12288 ms)."""
    net, onet = _line_net(orc, [512, 768, 0, 1536], [(0, 1, 512), (0, 2, 512), (1, 3, 768), (2, 3, 1536)])
    prep = orc.prepare(onet, orc.Params(), 3)
    assert list(prep["h"]) == [8192, 6144, 12288, 0]
    assert [int(net.col[e]) for e in range(net.row_ptr[0], net.row_ptr[1])] == [1, 2]
    tau = np.full(net.n_edges, 2**32, np.uint64)
    weights = _exact_weights([np.float32(2.0**-11), np.float32(2.0**-13)])
    assert weights == [2**22, 2**20]
    picks = []
    for ant in range(200):
        w = orc.walk_one(onet, orc.Params(), Q(0, 3, 200, 1, 1.0, 1.0, 0.1, 21), tau, it=0, ant=ant)
        pick = _expected_pick(orc, weights, 21, 0, ant, 0)
        assert [int(net.col[e]) for e in w["route_edges"]] == [[1, 3], [2, 3]][pick]
        assert w["T"] == [4096 + 6144, 4096 + 12288][pick] and w["moves"] == 2
        picks.append(pick)
    assert 0 < sum(picks) < 200


def test_hand_worked_cost_floor_at_one(orc):
    """A road that makes full progress at the fastest speed adds nothing over the bound: its cost is
    floored at 1 ms. src 0 at x = 512, node 1 at 1024, node 2 at 1536, destination 3 at 2048. The first
    move 0 -> 1 is forced. At 1 (h = 8192): road 1-2 of 512 dm gives c = 4096 + 4096 - 8192 = 0 -> 1,
    road 1-3 of 1025 dm (8200 ms) gives c = 8200 - 8192 = 8. Scores 1 and 1/8, weights 2^22 and 2^19:
    chances 8/9 and 1/9, drawn with the draw of move 1. The bound subtracted is the current node's
    (with src's, 12288, both costs would floor to 1)."""
    net, onet = _line_net(orc, [512, 1024, 1536, 2048], [(0, 1, 512), (1, 2, 512), (1, 3, 1025), (2, 3, 512)])
    assert [int(net.col[e]) for e in range(net.row_ptr[1], net.row_ptr[2])] == [0, 2, 3]
    tau = np.full(net.n_edges, 2**32, np.uint64)
    weights = _exact_weights([np.float32(1.0), np.float32(0.125)])
    assert weights == [2**22, 2**19]
    picks = []
    for ant in range(300):
        w = orc.walk_one(onet, orc.Params(), Q(0, 3, 300, 1, 1.0, 1.0, 0.1, 4), tau, it=0, ant=ant)
        pick = _expected_pick(orc, weights, 4, 0, ant, 1)
        assert [int(net.col[e]) for e in w["route_edges"]] == [[1, 2, 3], [1, 3]][pick]
        assert w["T"] == [4096 * 3, 4096 + 8200][pick]
        picks.append(pick)
    assert 0 < sum(picks) < 300


def _spur_junction():
    """Directed roads: 0 -> {1, 2, 3}, 1 -> 0 (node 1 is a dead end once 0 is visited), 2 -> {1, 4},
    3 -> 4; destination 4. Nodes 1, 2 and 3 are signalised, so every arrival time changes the waits
    that follow; an ant entering the dead end waits there (it arrives at 8400 ms, 3400 ms into the cycle,
    and its phase turns green at 20000 ms). All coordinates are equal (h = 0)."""
    roads = [(0, 1, 700, 30, 3, 1), (1, 0, 700, 30, 3, 0), (0, 2, 1200, 50, 3, 0), (0, 3, 900, 50, 3, 1),
             (2, 1, 800, 50, 3, 1), (2, 4, 1500, 70, 3, 0), (3, 4, 1300, 50, 3, 0)]
    signals = {1: (60_000, 5_000, [20_000, 40_000]), 2: (90_000, 30_000, [50_000, 40_000]),
               3: (75_000, 0, [30_000, 45_000])}
    return NB.build(5, roads, signals=signals, vehicles={(0, 2): 7, (2, 4): 3}, bidirectional=False)


def test_hand_worked_step_back_at_dead_end(orc):
    """Uniform choices (alpha = beta = 0). An ant that takes 0 -> 1 finds no unvisited node (1 -> 0 leads
    back), steps back to 0 with the clock and wait it had there, and draws again with the draw of move
    2 among {2, 3} (1 stays visited). An ant at 2 that takes 2 -> 1 steps back to 2 and must take 2 -> 4.
    Expected routes, move counts, T and W follow from the Philox draws and the pinned road times."""
    net, sig, veh = _spur_junction()
    onet = orc.Net(net, sig, veh)
    timing = NB.Timing(orc, onet, net, sig, 4)
    tau = np.full(net.n_edges, 2**32, np.uint64)

    def timed(route):
        t = Wt = 0
        for a, b in zip(route[:-1], route[1:]):
            t, w = timing.after(NB.edge_id(net, a, b), t)
            Wt += w
        return t, Wt

    seen = set()
    for ant in range(256):
        p0 = _expected_pick(orc, [1, 1, 1], 13, 0, ant, 0)
        if p0 == 0:  # into the dead end, back to 0, then 2 or 3 by the draw of move 2
            mid = [2, 3][_expected_pick(orc, [1, 1], 13, 0, ant, 2)]
            route, moves = [0, mid, 4], 4
        elif p0 == 1 and _expected_pick(orc, [1, 1], 13, 0, ant, 1) == 0:  # 0 -> 2 -> 1, back to 2, -> 4
            route, moves = [0, 2, 4], 4
        else:
            route, moves = [0, [1, 2, 3][p0], 4], 2
        w = orc.walk_one(onet, orc.Params(), Q(0, 4, 256, 1, 0.0, 0.0, 0.1, 13), tau, it=0, ant=ant)
        assert w["status"] == orc.ANT_SUCCESS
        assert [0] + [int(net.col[e]) for e in w["route_edges"]] == route, ant
        assert w["moves"] == moves and w["steps"] == 2
        assert (w["T"], w["W"]) == timed(route)
        seen.add((tuple(route), moves))
    assert len(seen) == 4  # both kinds of step back, and both direct routes, occurred
    assert timing.after(NB.edge_id(net, 0, 1), 0) == (8400 + 16600, 16600)


def _reachable(net, src):
    seen, stack = {src}, [src]
    while stack:
        u = stack.pop()
        for e in range(int(net.row_ptr[u]), int(net.row_ptr[u + 1])):
            v = int(net.col[e])
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return seen


@pytest.mark.parametrize("gseed", range(8))
def test_depth_first_walk_closed_forms(orc, gseed):
    """With the default cap of 2(N - 1) moves an ant is a depth-first search: it reaches any destination
    reachable from src, and when there is none it ends back at src with a dead end after exactly
    2(R - 1) moves, R = the number of nodes reachable from src (each is entered once and left once).
    Tree-like graphs with spurs, and directed graphs with sinks."""
    rng = np.random.Generator(np.random.PCG64(700 + gseed))
    n = int(rng.integers(6, 14))
    net, sig = W.random_small(n, n - 1 + int(rng.integers(0, 3)), rng, signalised_frac=0.5)
    if gseed % 2:  # keep one direction of a random half of the roads
        keep = rng.random(net.n_edges) < 0.6
        tails = net.tails()
        net = W.csr_from_roads(n, tails[keep], net.col[keep], net.length_dm[keep], net.speed_kmh[keep],
                               net.lanes[keep], net.orient[keep], net.x_dm, net.y_dm, bidirectional=False)
        sig = W.two_phase_signals(net, sig.n_phases > 0, rng)
    veh = rng.integers(0, 8, net.n_edges).astype(np.uint32)
    onet = orc.Net(net, sig, veh)
    src = 0
    R = _reachable(net, src)
    for dst in range(1, n):
        r = orc.solve(onet, orc.Params(), Q(src, dst, 8, 3, 1.0, 2.0, 0.1, gseed), want_tau=False, want_log=True)
        st, length, moves, _, _ = orc.log_fields(r["log"])
        if dst in R:
            assert (st == orc.ANT_SUCCESS).all() and r["status"] == 0
            assert (moves >= length).all() and ((moves - length) % 2 == 0).all()  # each step back undoes a move
        else:
            assert (st == orc.ANT_DEAD_END).all() and (moves == 2 * (len(R) - 1)).all() and (length == 0).all()
            assert r["status"] == orc.ERR_NO_ROUTE


@pytest.mark.parametrize("gseed", range(4))
def test_depth_first_walk_ignores_roads_to_themselves(orc, gseed):
    """The closed forms of the depth-first walk hold unchanged when every third node also has a road back
    to itself: such a road never becomes a way on, so an ant with no destination in reach still ends back
    at src after exactly 2(R - 1) moves, and one with a destination in reach still gets there."""
    rng = np.random.Generator(np.random.PCG64(900 + gseed))
    n = int(rng.integers(6, 14))
    base, _ = W.random_small(n, n - 1 + int(rng.integers(0, 3)), rng, signalised_frac=0.5)
    tails = base.tails()
    loops = np.arange(0, n, 3)
    net = W.csr_from_roads(n, np.concatenate([tails, loops]), np.concatenate([base.col, loops]),
                           np.concatenate([base.length_dm, np.full(loops.size, 300)]),
                           np.concatenate([base.speed_kmh, np.full(loops.size, 50)]),
                           np.concatenate([base.lanes, np.full(loops.size, 3)]),
                           np.concatenate([base.orient, np.zeros(loops.size, base.orient.dtype)]),
                           base.x_dm, base.y_dm, bidirectional=False)
    assert int((net.tails() == net.col).sum()) == loops.size
    sig = W.two_phase_signals(net, rng.random(n) < 0.5, rng)
    veh = rng.integers(0, 8, net.n_edges).astype(np.uint32)
    onet = orc.Net(net, sig, veh)
    R = _reachable(net, 0)
    for dst in range(1, n):
        r = orc.solve(onet, orc.Params(), Q(0, dst, 8, 3, 1.0, 2.0, 0.1, gseed), want_tau=False, want_log=True)
        st, length, moves, _, _ = orc.log_fields(r["log"])
        if dst in R:
            assert (st == orc.ANT_SUCCESS).all() and r["status"] == 0
            route = [int(v) for v in r["route"]]
            assert len(set(route)) == len(route)
        else:
            assert (st == orc.ANT_DEAD_END).all() and (moves == 2 * (len(R) - 1)).all() and (length == 0).all()


@pytest.mark.parametrize("gseed", range(6))
def test_spur_graphs_best_equals_brute_force(orc, gseed):
    """Trees with one or two extra links (many spurs and dead ends), signals at half the nodes: the
    colony's best route equals the time-dependent Dijkstra optimum and the brute-force minimum."""
    rng = np.random.Generator(np.random.PCG64(800 + gseed))
    net, sig = W.random_small(8, 8 + gseed % 2, rng, signalised_frac=0.5)
    veh = rng.integers(0, 10, net.n_edges).astype(np.uint32)
    onet = orc.Net(net, sig, veh)
    src, dst = 0, 7
    timing = NB.Timing(orc, onet, net, sig, dst)
    opt = NB.td_dijkstra(net, timing, src, dst)
    assert opt == NB.brute_force_min(net, timing, src, dst)
    r = orc.solve(onet, orc.Params(), Q(src, dst, 64, 30, 1.0, 2.0, 0.1, gseed))
    assert r["status"] == 0 and r["travel_ms"] == opt


def test_first_step_frequencies_chi_square(orc):
    """Scores 2^-12, 2^-13, 2^-11 -> probabilities 2/7, 1/7, 4/7 over Philox draws; and alpha=beta=0
    gives a uniform choice."""
    from scipy.stats import chisquare

    net, sig, veh = _star()
    onet = orc.Net(net, sig, veh)
    tau = np.full(net.n_edges, 2**32, np.uint64)
    for a, b, probs in [(1.0, 1.0, [2 / 7, 1 / 7, 4 / 7]), (0.0, 0.0, [1 / 3] * 3)]:
        counts = [0, 0, 0]
        n = 6000
        for ant in range(n):
            w = orc.walk_one(onet, orc.Params(), Q(0, 4, n, 1, a, b, 0.1, 5), tau, it=0, ant=ant)
            counts[int(net.col[w["route_edges"][0]]) - 1] += 1
        assert chisquare(counts, [n * p for p in probs]).pvalue > 1e-4, counts


@pytest.mark.parametrize("gseed", range(6))
def test_free_flow_best_equals_dijkstra_and_brute_force(orc, gseed):
    """No vehicles, no signals: the best colony route equals the shortest path (Dijkstra) and the
    minimum over all enumerated simple paths on tiny graphs."""
    rng = np.random.Generator(np.random.PCG64(100 + gseed))
    net, sig = W.random_small(7, 10, rng)
    veh = np.zeros(net.n_edges, np.uint32)
    onet = orc.Net(net, sig, veh)
    src, dst = 0, 6
    timing = NB.Timing(orc, onet, net, sig, dst)
    opt = NB.td_dijkstra(net, timing, src, dst)
    assert opt == NB.brute_force_min(net, timing, src, dst)
    r = orc.solve(onet, orc.Params(), Q(src, dst, 64, 30, 1.0, 2.0, 0.1, gseed))
    assert r["status"] == 0
    assert r["travel_ms"] == opt and r["wait_ms"] == 0


@pytest.mark.parametrize("gseed", range(6))
def test_signalised_best_equals_td_dijkstra_and_brute_force(orc, gseed):
    """Signals everywhere and random vehicles: waits are FIFO, so time-dependent Dijkstra is exact;
    the colony's best equals it and the brute-force minimum over simple paths."""
    rng = np.random.Generator(np.random.PCG64(200 + gseed))
    net, sig = W.random_small(7, 11, rng, signalised_frac=1.0)
    veh = rng.integers(0, 12, net.n_edges).astype(np.uint32)
    onet = orc.Net(net, sig, veh)
    src, dst = 1, 5
    timing = NB.Timing(orc, onet, net, sig, dst)
    opt = NB.td_dijkstra(net, timing, src, dst)
    assert opt == NB.brute_force_min(net, timing, src, dst)
    r = orc.solve(onet, orc.Params(), Q(src, dst, 64, 40, 1.0, 2.0, 0.1, gseed))
    assert r["status"] == 0
    assert r["travel_ms"] == opt


def _check_route(orc, net, sig, onet, res, q, params=None):
    route = [int(v) for v in res["route"]]
    assert route[0] == q.src and route[-1] == q.dst
    assert len(set(route)) == len(route)
    timing = NB.Timing(orc, onet, net, sig, q.dst, params)
    t = Wt = 0
    for u, v in zip(route[:-1], route[1:]):
        e = NB.edge_id(net, u, v)
        t, w = timing.after(e, t)
        Wt += w
    assert t == res["travel_ms"] and Wt == res["wait_ms"] and Wt <= t


def test_grid10_route_validity_and_recomputed_times(orc):
    wl = W.grid10()
    onet = orc.Net.from_workload(wl)
    q = wl.queries[0]
    r = orc.solve(onet, orc.Params(), q)
    assert r["status"] == 0
    _check_route(orc, wl.net, wl.signals, onet, r, q)
    # departure clock shifts signal phases but the route stays valid and timed consistently
    p = orc.Params(t_dep_ms=123_457)
    r2 = orc.solve(onet, p, q)
    _check_route(orc, wl.net, wl.signals, onet, r2, q, p)


def test_grid64_full_size_best_routes_valid_and_bounded(orc):
    """Properties that hold at any size, on two benchmark colonies at full size (1024 ants x 200
    iterations; colony 11 has the job's longest walks): the best route is a simple path from src to dst
    along roads; its travel and wait times, recomputed road by road from the pinned primitives, equal
    the reported ones; and it is no faster than the time-dependent Dijkstra optimum (waits are FIFO, so
    that optimum is exact)."""
    wl = W.grid64()
    onet = orc.Net.from_workload(wl)
    for qi in (0, 11):
        q = wl.queries[qi]
        r = orc.solve(onet, orc.Params(), q, want_tau=False)
        assert r["status"] == 0 and r["n_success"] > 0
        _check_route(orc, wl.net, wl.signals, onet, r, q)
        timing = NB.Timing(orc, onet, wl.net, wl.signals, q.dst)
        opt = NB.td_dijkstra(wl.net, timing, q.src, q.dst)
        assert opt is not None and r["travel_ms"] >= opt


def _deposit(h_src, T):
    return (max(h_src, 1) << 32) // T


def test_pheromone_conservation_identity(orc):
    """sum tau' = sum (tau - floor(tau*rho_fix/2^32)) + sum over successful ants of |route| * delta."""
    wl = W.grid10(n_ants=32, n_iter=1)
    onet = orc.Net.from_workload(wl)
    q = wl.queries[0]
    h_src = int(orc.prepare(onet, orc.Params(), q.dst)["h"][q.src])
    rfix = orc.rho_fix(q.rho)
    r1 = orc.solve(onet, orc.Params(), q, want_log=True)
    log = r1["log"][0]
    st, length, _, T, _ = orc.log_fields(log)
    dep = sum(int(n) * _deposit(h_src, int(t)) for n, t in zip(length[st == 0], T[st == 0]))
    assert dep > 0
    E = wl.net.n_edges
    assert int(r1["tau"].sum()) == E * orc.evaporate(2**32, rfix) + dep
    assert r1["ant_steps"] == int(log[:, 1].sum())
    # second iteration, starting from the first iteration's table (deterministic prefix)
    q2 = W.Query(q.src, q.dst, q.n_ants, 2, q.alpha, q.beta, q.rho, q.seed)
    r2 = orc.solve(onet, orc.Params(), q2, want_log=True)
    assert (r2["log"][0] == log).all()
    st2, length2, _, T2, _ = orc.log_fields(r2["log"][1])
    dep2 = sum(int(n) * _deposit(h_src, int(t)) for n, t in zip(length2[st2 == 0], T2[st2 == 0]))
    assert int(r2["tau"].sum()) == sum(orc.evaporate(int(t), rfix) for t in r1["tau"]) + dep2
    assert int(r2["tau"].min()) >= 1


def _star_solve(orc):
    net, sig, veh = _star()
    return orc.solve(orc.Net(net, sig, veh), orc.Params(), Q(0, 4, 16, 4, 1.0, 2.0, 0.1, 3), want_log=True)


def _grid_solve(orc):
    wl = W.grid10(n_ants=16, n_iter=6)
    return orc.solve(orc.Net.from_workload(wl), orc.Params(), wl.queries[0], want_log=True)


@pytest.mark.parametrize("case", ["star", "grid10"])
def test_best_is_min_T_then_lowest_iteration_ant(orc, case):
    """The reported best is the minimum T; among equal T (many on the star graph), the lowest
    (iteration, ant)."""
    r = _star_solve(orc) if case == "star" else _grid_solve(orc)
    st, length, _, T, W_ = orc.log_fields(r["log"])
    ok = st == 0
    Ts = np.where(ok, T.astype(np.int64), np.iinfo(np.int64).max)
    tmin = Ts.min()
    it, ant = [int(v) for v in np.argwhere(Ts == tmin)[0]]  # row-major: lowest (it, ant)
    assert r["travel_ms"] == tmin and (r["best_iter"], r["best_ant"]) == (it, ant)
    assert r["wait_ms"] == W_[it, ant] and r["route_len"] == length[it, ant] + 1
    assert r["n_success"] == int(ok.sum())
    if case == "star":
        assert (Ts == tmin).sum() > 10


def test_src_equals_dst(orc):
    wl = W.grid10()
    onet = orc.Net.from_workload(wl)
    r = orc.solve(onet, orc.Params(), Q(5, 5, 8, 3, 1.0, 2.0, 0.1, 0))
    assert r["status"] == 0 and list(r["route"]) == [5] and r["travel_ms"] == 0 and r["ant_steps"] == 0
    assert (r["tau"] == 2**32).all()


def test_unreachable_destination(orc):
    """Node 3 is isolated. Every ant walks 0 -> 1 -> 2, finds no road left, steps back twice and ends at
    src with nothing left to try: 4 moves, a dead end, no route."""
    net, sig, veh = NB.build(4, [(0, 1, 1000, 50), (1, 2, 1000, 50)])  # node 3 isolated
    r = orc.solve(orc.Net(net, sig, veh), orc.Params(), Q(0, 3, 8, 4, 1.0, 2.0, 0.1, 0), want_log=True)
    assert r["status"] == orc.ERR_NO_ROUTE
    st, length, moves, _, _ = orc.log_fields(r["log"])
    assert set(np.unique(st)) == {orc.ANT_DEAD_END} and (moves == 4).all() and (length == 0).all()
    assert r["ant_steps"] == 4 * 8 * 4


def test_step_cap(orc):
    roads = [(i, i + 1, 1000, 50) for i in range(6)]
    net, sig, veh = NB.build(7, roads)
    onet = orc.Net(net, sig, veh)
    r = orc.solve(onet, orc.Params(max_steps=5), Q(0, 6, 4, 2, 1.0, 2.0, 0.1, 0), want_log=True)
    assert r["status"] == orc.ERR_NO_ROUTE
    st, length, moves, _, _ = orc.log_fields(r["log"])
    assert (st == orc.ANT_STEP_CAP).all() and (moves == 5).all() and (length == 5).all()
    r = orc.solve(onet, orc.Params(max_steps=6), Q(0, 6, 4, 2, 1.0, 2.0, 0.1, 0))
    assert r["status"] == 0 and r["route_len"] == 7


def test_default_step_cap_is_4096(orc):
    """With max_steps = 0 the cap is min(2(N - 1), 4096) moves (Q12's reading). On a line of 4200 nodes
    the only walk from one end to the other has 4199 roads, so it stops after exactly 4096; with the
    cap raised to 4199 it arrives."""
    roads = [(i, i + 1, 1000, 50) for i in range(4199)]
    net, sig, veh = NB.build(4200, roads)
    onet = orc.Net(net, sig, veh)
    q = Q(0, 4199, 2, 1, 1.0, 2.0, 0.1, 0)
    r = orc.solve(onet, orc.Params(), q, want_log=True)
    assert r["status"] == orc.ERR_NO_ROUTE
    st, _, moves, _, _ = orc.log_fields(r["log"])
    assert (st == orc.ANT_STEP_CAP).all() and (moves == 4096).all()
    r = orc.solve(onet, orc.Params(max_steps=4199), q)
    assert r["status"] == 0 and r["route_len"] == 4200


def test_time_cap(orc):
    """Roads whose free-flow time clamps at 2^26 ms: 16 of them take exactly 2^30 ms (allowed),
    the 17th exceeds the 2^30 ms cap and the ant fails."""
    roads = [(i, i + 1, 10**9, 1) for i in range(17)]
    net, sig, veh = NB.build(18, roads)
    onet = orc.Net(net, sig, veh)
    r = orc.solve(onet, orc.Params(), Q(0, 16, 2, 1, 1.0, 2.0, 0.1, 0))
    assert r["status"] == 0 and r["travel_ms"] == 2**30
    r = orc.solve(onet, orc.Params(), Q(0, 17, 2, 1, 1.0, 2.0, 0.1, 0), want_log=True)
    assert r["status"] == orc.ERR_NO_ROUTE and (orc.log_fields(r["log"])[0] == orc.ANT_TIME_CAP).all()


def test_congestion_threshold_mask(orc):
    """Fig. 3's threshold: a road over the occupancy threshold is avoided unless all are over."""
    # 0 -> 1 (congested: 30 of cap 40), 0 -> 2 (empty); both lead to 3
    roads = [(0, 1, 1000, 50), (0, 2, 1000, 50), (1, 3, 1000, 50), (2, 3, 1000, 50)]
    net, sig, veh = NB.build(4, roads, vehicles={(0, 1): 30})
    onet = orc.Net(net, sig, veh)
    tau = np.full(net.n_edges, 2**32, np.uint64)
    p = orc.Params(thr_permille=500)  # over half full counts as congested
    firsts = {int(net.col[orc.walk_one(onet, p, Q(0, 3, 64, 1, 0.0, 0.0, 0.1, 1), tau, 0, k)["route_edges"][0]])
              for k in range(64)}
    assert firsts == {2}
    # both congested -> both allowed again
    net, sig, veh = NB.build(4, roads, vehicles={(0, 1): 30, (0, 2): 35})
    onet = orc.Net(net, sig, veh)
    firsts = {int(net.col[orc.walk_one(onet, p, Q(0, 3, 64, 1, 0.0, 0.0, 0.1, 1), tau, 0, k)["route_edges"][0]])
              for k in range(64)}
    assert firsts == {1, 2}


def test_invalid_and_unsupported_queries(orc):
    wl = W.grid10()
    onet = orc.Net.from_workload(wl)
    assert orc.solve(onet, orc.Params(), Q(0, 99, 8, 2, 8.5, 2.0, 0.1, 0))["status"] == orc.ERR_UNSUPPORTED
    assert orc.solve(onet, orc.Params(), Q(0, 99, 8, 2, 1.0, -0.5, 0.1, 0))["status"] == orc.ERR_UNSUPPORTED
    assert orc.solve(onet, orc.Params(), Q(0, 99, 8, 2, float("nan"), 2.0, 0.1, 0))["status"] == orc.ERR_UNSUPPORTED
    assert orc.solve(onet, orc.Params(), Q(0, 99, 8, 2, 1.0, 2.0, 1.0, 0))["status"] == orc.ERR_INVALID
    assert orc.solve(onet, orc.Params(), Q(0, 100, 8, 2, 1.0, 2.0, 0.1, 0))["status"] == orc.ERR_INVALID
    assert orc.solve(onet, orc.Params(), Q(0, 99, 0, 2, 1.0, 2.0, 0.1, 0))["status"] == orc.ERR_INVALID
    r = orc.solve(onet, orc.Params(), wl.queries[0], route_cap=3)
    assert r["status"] == orc.ERR_BUFFER and r["route_len"] > 3


def test_queue_preempt_on_network(orc):
    """Per-phase queues add up the vehicles on each phase's approaches; a queue over 3/4 of the
    approach storage is preempted first."""
    # node 2 signalised with 3 phases; approaches 0->2 (phase 0), 1->2 (phase 1), 3->2 (phase 2)
    roads = [(0, 2, 1000, 50, 3, 0), (1, 2, 1000, 50, 3, 1), (3, 2, 1000, 50, 3, 2)]
    sigs = {2: (90_000, 0, [30_000, 30_000, 30_000])}
    # capacities 40 each -> threshold 30. queues 5, 0, 12: no preemption -> longest (2) first,
    # then non-empty in default order (0), then empty (1)
    net, sig, veh = NB.build(4, roads, signals=sigs, vehicles={(0, 2): 5, (3, 2): 12}, bidirectional=False)
    sig.edge_phase[:] = net.orient
    assert list(orc.queue_preempt(orc.Net(net, sig, veh))[2][:3]) == [2, 0, 1]
    # queue 31 on phase 1 exceeds its threshold 30
    net, sig, veh = NB.build(4, roads, signals=sigs, vehicles={(0, 2): 5, (1, 2): 31, (3, 2): 12},
                             bidirectional=False)
    assert list(orc.queue_preempt(orc.Net(net, sig, veh))[2][:3]) == [1, 0, 2]
    # red accumulator above T_max (= cycle) on phase 0 with no queue over threshold
    red = np.zeros((4, 8), np.uint32)
    red[2, 0] = 90_001
    net, sig, veh = NB.build(4, roads, signals=sigs, vehicles={(0, 2): 5, (3, 2): 12}, bidirectional=False)
    assert list(orc.queue_preempt(orc.Net(net, sig, veh, red))[2][:3]) == [0, 2, 1]
    # queue 25 on phase 0 lies between half (20) and three quarters (30) of its storage: no
    # preemption by queue, so the starved phase 2 goes first
    red[2, 0] = 0
    red[2, 2] = 90_001
    net, sig, veh = NB.build(4, roads, signals=sigs, vehicles={(0, 2): 25, (3, 2): 12}, bidirectional=False)
    assert list(orc.queue_preempt(orc.Net(net, sig, veh, red))[2][:3]) == [2, 0, 1]


def test_roads_from_a_node_to_itself_are_never_taken(orc):
    """A road from a node back to itself is never a way on: the node is visited from the moment the ant
    stands on it. On a ring-and-chord graph where every third node carries such a road, the best routes are
    simple paths whose times recompute road by road, and no such road ever receives a deposit: its final
    pheromone is 1.0 evaporated once per iteration, exactly."""
    rng = np.random.default_rng(23)
    roads = []
    for u in range(48):
        for v in ((u + 1) % 48, (u + 7) % 48):
            L = int(rng.integers(300, 3000))
            roads += [(u, v, L, 50, 3, 0), (v, u, L, 50, 3, 1)]
    for u in range(0, 48, 3):
        roads.append((u, u, int(rng.integers(100, 400)), 50, 3, 0))
    sigs = {v: (30_000, int(rng.integers(0, 30_000)), [18_000, 12_000]) for v in range(0, 48, 5)}
    net, sig, veh = NB.build(48, roads, signals=sigs, bidirectional=False)
    veh[:] = rng.integers(0, 20, size=veh.size)
    onet = orc.Net(net, sig, veh)
    loops = np.flatnonzero(net.tails() == net.col)
    assert loops.size == 16
    for i, (s, d) in enumerate([(0, 47), (3, 30), (9, 21)]):
        q = Q(s, d, 40, 6, 1.0, 2.0, 0.1, 300 + i)
        r = orc.solve(onet, orc.Params(), q)
        assert r["status"] == 0
        _check_route(orc, net, sig, onet, r, q)
        rho_fix = round(float(np.float32(q.rho)) * 2**32)  # the query's rho is binary32
        tau = 1 << 32
        for _ in range(q.n_iter):
            tau -= (tau * rho_fix) >> 32
        assert (np.asarray(r["tau"])[loops] == tau).all()

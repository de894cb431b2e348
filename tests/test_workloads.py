"""The seeded synthetic inputs: each generator against the recipe it states (sizes, value ranges,
distributions, structure), and every generator is deterministic. No GPU."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components, shortest_path

from paper_2010_14244_gb300 import workloads as W


def _csr_ok(net):
    rp = net.row_ptr.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == net.n_edges and np.all(np.diff(rp) >= 0)
    assert net.col.min() >= 0 and net.col.max() < net.n_nodes
    tails = net.tails()
    assert np.all(tails != net.col)  # no self-loops
    keys = tails.astype(np.int64) * net.n_nodes + net.col
    assert np.unique(keys).size == keys.size  # no parallel roads


def _strongly_connected(net):
    adj = csr_matrix((np.ones(net.n_edges), net.col.astype(np.int64), net.row_ptr.astype(np.int64)),
                     shape=(net.n_nodes, net.n_nodes))
    return connected_components(adj, directed=True, connection="strong")[0] == 1


def _signals_ok(sig, net, signalised):
    P = sig.n_phases.astype(np.int64)
    assert set(np.unique(P[signalised])) <= {2} and np.all(P[~signalised] == 0)
    green = sig.green_ms.reshape(net.n_nodes, 8).astype(np.int64)
    cyc = sig.cycle_ms.astype(np.int64)
    s = signalised
    assert np.all(cyc[s] % 1000 == 0) and cyc[s].min() >= 60_000 and cyc[s].max() <= 120_000
    assert np.all(green[s, 0] + green[s, 1] == cyc[s]) and np.all(green[s, 2:] == 0)
    split = green[s, 0] * 100 // cyc[s]  # phase 0's share, U{30..70} %
    assert split.min() >= 30 and split.max() <= 70
    assert np.all(sig.offset_ms.astype(np.int64)[s] < cyc[s])
    np.testing.assert_array_equal(sig.edge_phase, net.orient)  # horizontal approaches phase 0, vertical 1


def test_grid10_recipe():
    wl = W.grid10()
    net = wl.net
    assert net.n_nodes == 100 and net.n_edges == 360
    _csr_ok(net)
    assert _strongly_connected(net)
    L = net.length_dm.astype(np.int64)
    assert L.min() >= 1000 and L.max() <= 5000
    assert set(np.unique(net.speed_kmh).tolist()) <= {30, 50, 70} and np.all(net.lanes == 3)
    _signals_ok(wl.signals, net, np.ones(100, bool))
    assert int(wl.vehicles.sum()) == 200
    (q,) = wl.queries
    assert (q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed) == (0, 99, 32, 50, 1.0, 2.0, 0.1, 0)
    # node spacing equals the shortest road, so the straight line never exceeds a road path
    tails = net.tails()
    d = np.hypot(net.x_dm[tails] - net.x_dm[net.col], net.y_dm[tails] - net.y_dm[net.col])
    assert np.all(d <= L)


def test_grid64_recipe():
    wl = W.grid64()
    net = wl.net
    assert net.n_nodes == 4096 and net.n_edges == 14916
    _csr_ok(net)
    assert _strongly_connected(net)
    deg = np.diff(net.row_ptr.astype(np.int64))
    assert deg.max() == 6 and abs(net.n_edges / net.n_nodes - 3.64) < 0.01
    tails = net.tails().astype(np.int64)
    head = net.col.astype(np.int64)
    dr, dc = np.abs(tails // 64 - head // 64), np.abs(tails % 64 - head % 64)
    grid = dr + dc == 1
    # 10 % of the 8064 grid road pairs removed: 7258 pairs kept, both directions
    assert int(grid.sum()) == 2 * 7258
    # 200 arterials, both directions: straight along a row or column, 4..16 cells, length = the distance,
    # speed 1.5 x a grid limit
    art = ~grid
    assert int(art.sum()) == 400
    span = np.where(dr[art] == 0, dc[art], dr[art])
    assert np.all((dr[art] == 0) | (dc[art] == 0)) and span.min() >= 4 and span.max() <= 16
    np.testing.assert_array_equal(net.length_dm[art].astype(np.int64), span * 1000)
    assert set(np.unique(net.speed_kmh[art]).tolist()) <= {45, 75, 105}
    _signals_ok(wl.signals, net, np.ones(4096, bool))
    assert int(wl.vehicles.sum()) == 2000
    # rank-Zipf(1.2): the most loaded road carries far more than a uniform placement would give
    assert int(wl.vehicles.max()) > 100 and np.count_nonzero(wl.vehicles) < 1000
    assert len(wl.queries) == 16 and len({(q.src, q.dst) for q in wl.queries}) == 16
    for i, q in enumerate(wl.queries):
        assert q.src != q.dst and (q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed) == (1024, 200, 1.0, 2.0, 0.1, i)


def test_geo100k_recipe():
    wl = W.geo100k(n_queries=16)
    net = wl.net
    assert net.n_nodes == 100_000
    _csr_ok(net)
    assert abs(net.n_edges / net.n_nodes - 2.8) < 0.005
    # planar lattice links only (4-neighbour), both directions, connected
    tails = net.tails().astype(np.int64)
    head = net.col.astype(np.int64)
    dr, dc = np.abs(tails // 400 - head // 400), np.abs(tails % 400 - head % 400)
    assert np.all(dr + dc == 1)
    assert _strongly_connected(net)
    # length = straight-line distance x U[1.0, 1.4], rounded up
    d = np.hypot((net.x_dm[tails] - net.x_dm[head]).astype(np.float64),
                 (net.y_dm[tails] - net.y_dm[head]).astype(np.float64))
    L = net.length_dm.astype(np.float64)
    assert np.all(L >= np.floor(d)) and np.all(L <= np.ceil(d * 1.4) + 1)
    frac = np.count_nonzero(wl.signals.n_phases) / net.n_nodes
    assert abs(frac - 0.6) < 0.01
    _signals_ok(wl.signals, net, wl.signals.n_phases > 0)
    assert abs(float(wl.vehicles.mean()) - 1.0) < 0.02  # Poisson(1) per road
    # OD pairs with BFS hop counts 20..400
    adj = csr_matrix((np.ones(net.n_edges), head, net.row_ptr.astype(np.int64)), shape=(net.n_nodes,) * 2)
    for q in wl.queries[:6]:
        hops = shortest_path(adj, method="D", unweighted=True, indices=q.src)[q.dst]
        assert 20 <= hops <= 400
    assert all((q.n_ants, q.n_iter) == (256, 100) for q in wl.queries)


def _thin_literally(n, a, b, order, target):
    """The recipe as stated: try the links in `order`; remove a link when it is not a bridge of what
    remains (the graph stays connected without it); stop when `target` links remain."""
    import networkx as nx

    g = nx.MultiGraph()
    g.add_nodes_from(range(n))
    for i, (p, q) in enumerate(zip(a, b)):
        g.add_edge(int(p), int(q), key=i)
    kept = set(range(len(a)))
    for i in order:
        if len(kept) == target:
            break
        g.remove_edge(int(a[i]), int(b[i]), key=int(i))
        if nx.is_connected(g):
            kept.discard(int(i))
        else:
            g.add_edge(int(a[i]), int(b[i]), key=int(i))
    return np.array(sorted(kept))


@pytest.mark.parametrize("seed", range(6))
def test_thin_lattice_equals_one_at_a_time_removal(seed):
    """The spanning-tree form of the planar generator keeps exactly the links that removing random
    non-bridge links one at a time keeps, for the same order of tries."""
    rng = np.random.default_rng(seed)
    rows, cols = int(rng.integers(3, 8)), int(rng.integers(3, 9))
    n = rows * cols
    ids = np.arange(n).reshape(rows, cols)
    a = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    b = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    order = rng.permutation(a.size)
    for target in (n - 1, int(round(1.2 * n)), int(round(1.4 * n)), a.size):
        target = min(target, a.size)
        np.testing.assert_array_equal(W.thin_lattice(n, a, b, order, target), _thin_literally(n, a, b, order, target))


def test_city52_recipe():
    wl = W.city52()
    net = wl.net
    assert net.n_nodes == 52 and net.n_edges == 128 and np.all(net.lanes == 3)
    _csr_ok(net)
    assert _strongly_connected(net)
    streets = np.diff(net.row_ptr.astype(np.int64))  # two-way streets: out-degree = streets at the node
    _signals_ok(wl.signals, net, streets >= 3)
    assert int(wl.vehicles.sum()) == 0


@pytest.mark.parametrize("make", [W.grid10, W.grid64, W.city52, lambda: W.geo100k(n_queries=4)])
def test_generators_are_deterministic(make):
    a, b = make(), make()
    for f in ("row_ptr", "col", "length_dm", "speed_kmh", "lanes", "x_dm", "y_dm", "orient"):
        np.testing.assert_array_equal(getattr(a.net, f), getattr(b.net, f))
    for f in ("n_phases", "cycle_ms", "offset_ms", "green_ms", "edge_phase"):
        np.testing.assert_array_equal(getattr(a.signals, f), getattr(b.signals, f))
    np.testing.assert_array_equal(a.vehicles, b.vehicles)
    assert a.queries == b.queries


def test_city_batch_recipe():
    """64 independent city graphs: node counts log-uniform in [1k, 200k] from the same planar generator,
    60 % signalised, mean density U[0.5, 3] vehicles per road, 8-64 uniform OD queries of 128-1024 ants."""
    cities = W.city_batch()
    assert len(cities) == 64
    ns = np.array([wl.net.n_nodes for wl in cities])
    assert ns.min() >= 900 and ns.max() <= 200_000
    logs = np.log(ns)
    assert logs.std() > 0.8  # spread over the decades, not clustered
    for wl in cities:
        net = wl.net
        _csr_ok(net)
        assert abs(net.n_edges / net.n_nodes - 2.8) < 0.05
        assert 8 <= len(wl.queries) <= 64
        assert all(128 <= q.n_ants <= 1024 and q.n_iter == 50 and q.src != q.dst for q in wl.queries)
        assert 0.4 <= float(wl.vehicles.mean()) <= 3.2
        frac = np.count_nonzero(wl.signals.n_phases) / net.n_nodes
        assert abs(frac - 0.6) < 0.08
    assert sum(len(wl.queries) for wl in cities) == 2362


def test_serving_requests():
    """Uniform OD requests, src != dst, 128 ants x 30 iterations; request i's seed is
    1,000,003 * i + the stream seed, so every request has its own Philox key."""
    from paper_2010_14244_gb300 import serving

    make = serving.uniform_requests(1000, 128, 30, seed=5)
    qs = [make(i) for i in range(4000)]
    assert all(q.src != q.dst and 0 <= q.src < 1000 and 0 <= q.dst < 1000 for q in qs)
    assert all((q.n_ants, q.n_iter, q.alpha, q.beta, q.rho) == (128, 30, 1.0, 2.0, 0.1) for q in qs)
    assert [q.seed for q in qs[:3]] == [5, 1_000_008, 2_000_011]
    counts = np.bincount([q.src for q in qs], minlength=1000)
    assert counts.max() < 16  # uniform: about 4 per node
    again = serving.uniform_requests(1000, 128, 30, seed=5)
    assert [again(i) for i in range(50)] == qs[:50]

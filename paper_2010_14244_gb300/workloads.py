"""Seeded synthetic road-network workloads.

This module only *draws inputs*: graph topology, road attributes (length, speed limit, lanes), node
coordinates, fixed-time signal timing, vehicle counts per road and origin-destination queries. It holds
none of the route-colony arithmetic (no travel times, capacities, waits, scores or pheromone): the CUDA
path and the CPU oracle each derive those from these raw inputs on their own.

The paper's experiment network (52 intersections / 128 roads / 3 lanes, Sec. 5) is not available, so
these generators stand in for it with grids and planar geometric graphs of the sizes and value
distributions listed per workload below. Every draw is made with ``numpy.random.Generator(PCG64(seed))``.

Units: lengths and coordinates in decimetres (int), speeds in km/h (int), times in milliseconds (int).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAX_PHASES = 8
SPEEDS_KMH = (30, 50, 70)


@dataclass
class RoadNetwork:
    """Directed road graph in CSR form (edges grouped by tail node, ascending head within a tail)."""

    row_ptr: np.ndarray  # uint32 [N+1]
    col: np.ndarray  # uint32 [E] head node of each directed road
    length_dm: np.ndarray  # uint32 [E]
    speed_kmh: np.ndarray  # uint16 [E]
    lanes: np.ndarray  # uint8  [E]
    x_dm: np.ndarray  # int32  [N]
    y_dm: np.ndarray  # int32  [N]
    orient: np.ndarray  # uint8 [E] 0 = mostly horizontal road, 1 = mostly vertical (drives edge_phase)

    @property
    def n_nodes(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n_edges(self) -> int:
        return int(self.col.shape[0])

    def tails(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_nodes, dtype=np.uint32), np.diff(self.row_ptr).astype(np.int64))


@dataclass
class SignalTiming:
    """Fixed-time signal programme per node; n_phases == 0 marks an unsignalised node."""

    n_phases: np.ndarray  # uint8  [N]
    cycle_ms: np.ndarray  # uint32 [N]
    offset_ms: np.ndarray  # uint32 [N]
    green_ms: np.ndarray  # uint32 [N*8], phase p of node v at v*8+p; sums to cycle_ms
    edge_phase: np.ndarray  # uint8 [E] approach phase of each road at its head node


@dataclass
class Query:
    src: int
    dst: int
    n_ants: int
    n_iter: int
    alpha: float
    beta: float
    rho: float
    seed: int


@dataclass
class Workload:
    name: str
    net: RoadNetwork
    signals: SignalTiming
    vehicles: np.ndarray  # uint32 [E] vehicles currently on each road
    queries: list[Query] = field(default_factory=list)
    description: str = ""


# ----------------------------------------------------------------------------------------------
# graph construction helpers
# ----------------------------------------------------------------------------------------------
def csr_from_roads(n_nodes, a, b, length_dm, speed_kmh, lanes, orient, x_dm, y_dm,
                   bidirectional=True) -> RoadNetwork:
    """Build the CSR network from an undirected (or directed) road list."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    length_dm = np.asarray(length_dm, dtype=np.int64)
    speed_kmh = np.asarray(speed_kmh, dtype=np.int64)
    lanes = np.asarray(lanes, dtype=np.int64)
    orient = np.asarray(orient, dtype=np.int64)
    if bidirectional:
        tail = np.concatenate([a, b])
        head = np.concatenate([b, a])
        length_dm, speed_kmh, lanes, orient = (np.concatenate([v, v]) for v in (length_dm, speed_kmh, lanes, orient))
    else:
        tail, head = a, b
    order = np.lexsort((length_dm, head, tail))
    tail, head = tail[order], head[order]
    counts = np.bincount(tail, minlength=n_nodes)
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return RoadNetwork(
        row_ptr=row_ptr.astype(np.uint32),
        col=head.astype(np.uint32),
        length_dm=length_dm[order].astype(np.uint32),
        speed_kmh=speed_kmh[order].astype(np.uint16),
        lanes=lanes[order].astype(np.uint8),
        x_dm=np.asarray(x_dm, dtype=np.int32),
        y_dm=np.asarray(y_dm, dtype=np.int32),
        orient=orient[order].astype(np.uint8),
    )


def _connected(n_nodes, a, b) -> bool:
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    m = coo_matrix((np.ones(len(a)), (np.asarray(a), np.asarray(b))), shape=(n_nodes, n_nodes))
    n_comp, _ = connected_components(m, directed=False)
    return n_comp == 1


def grid_roads(rows, cols, rng, spacing_dm=1000, len_lo=1000, len_hi=5000):
    """4-neighbour grid. Returns undirected roads (a, b, length, speed, orient) and coordinates.

    The node spacing equals the minimum road length, so the straight-line distance between any two
    nodes never exceeds the length of a road path joining them.
    """
    ids = np.arange(rows * cols).reshape(rows, cols)
    ha, hb = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    va, vb = ids[:-1, :].ravel(), ids[1:, :].ravel()
    a = np.concatenate([ha, va])
    b = np.concatenate([hb, vb])
    orient = np.concatenate([np.zeros(ha.size, np.int64), np.ones(va.size, np.int64)])
    length = rng.integers(len_lo, len_hi + 1, size=a.size)
    speed = rng.choice(np.array(SPEEDS_KMH), size=a.size)
    x = (np.arange(rows * cols) % cols) * spacing_dm
    y = (np.arange(rows * cols) // cols) * spacing_dm
    return a, b, length, speed, orient, x, y


def two_phase_signals(net: RoadNetwork, signalised: np.ndarray, rng) -> SignalTiming:
    """Two-phase fixed-time signals: phase 0 serves horizontal approaches, phase 1 vertical ones.

    cycle ~ U{60..120} s, green split of phase 0 ~ U{0.30..0.70} in steps of 0.01, offset ~ U[0, cycle).
    """
    n = net.n_nodes
    cycle = rng.integers(60, 121, size=n).astype(np.int64) * 1000
    split = rng.integers(30, 71, size=n).astype(np.int64)
    offset = (rng.random(n) * cycle).astype(np.int64)
    g0 = cycle * split // 100
    g1 = cycle - g0
    sig = np.asarray(signalised, dtype=bool)
    green = np.zeros((n, MAX_PHASES), dtype=np.int64)
    green[:, 0] = np.where(sig, g0, 0)
    green[:, 1] = np.where(sig, g1, 0)
    return SignalTiming(
        n_phases=np.where(sig, 2, 0).astype(np.uint8),
        cycle_ms=np.where(sig, cycle, 0).astype(np.uint32),
        offset_ms=np.where(sig, offset, 0).astype(np.uint32),
        green_ms=green.ravel().astype(np.uint32),
        edge_phase=net.orient.astype(np.uint8).copy(),
    )


def vehicles_uniform(n_edges, n_vehicles, rng) -> np.ndarray:
    return np.bincount(rng.integers(0, n_edges, size=n_vehicles), minlength=n_edges).astype(np.uint32)


def vehicles_zipf(n_edges, n_vehicles, s, rng) -> np.ndarray:
    """Rank-Zipf(s) vehicle placement over a random permutation of the roads."""
    ranks = np.arange(1, n_edges + 1, dtype=np.float64)
    p = ranks ** (-s)
    p /= p.sum()
    perm = rng.permutation(n_edges)
    picks = rng.choice(n_edges, size=n_vehicles, p=p)
    return np.bincount(perm[picks], minlength=n_edges).astype(np.uint32)


def vehicles_poisson(n_edges, mean, rng) -> np.ndarray:
    return rng.poisson(mean, size=n_edges).astype(np.uint32)


def uniform_od(n_nodes, n_pairs, rng):
    out = []
    while len(out) < n_pairs:
        s, d = (int(v) for v in rng.integers(0, n_nodes, size=2))
        if s != d:
            out.append((s, d))
    return out


def hop_filtered_od(net: RoadNetwork, n_pairs, lo, hi, rng):
    """Uniform OD pairs whose BFS hop count lies in [lo, hi]."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path

    n = net.n_nodes
    adj = csr_matrix((np.ones(net.n_edges), net.col.astype(np.int64), net.row_ptr.astype(np.int64)), shape=(n, n))
    out = []
    while len(out) < n_pairs:
        s = int(rng.integers(0, n))
        hops = shortest_path(adj, method="D", unweighted=True, indices=s)
        ok = np.flatnonzero((hops >= lo) & (hops <= hi) & np.isfinite(hops))
        if ok.size == 0:
            continue
        out.append((s, int(ok[rng.integers(0, ok.size)])))
    return out


# ----------------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------------
def grid10(n_ants=32, n_iter=50) -> Workload:
    """10x10 grid, 360 directed roads, signals everywhere, 200 uniform vehicles, OD corner to corner."""
    rng = np.random.Generator(np.random.PCG64(1))
    a, b, length, speed, orient, x, y = grid_roads(10, 10, rng)
    net = csr_from_roads(100, a, b, length, speed, np.full(a.size, 3), orient, x, y)
    sig = two_phase_signals(net, np.ones(100, bool), rng)
    veh = vehicles_uniform(net.n_edges, 200, rng)
    q = [Query(0, 99, n_ants, n_iter, 1.0, 2.0, 0.1, 0)]
    return Workload("grid10", net, sig, veh, q,
                    "10x10 grid, 360 roads, 3 lanes, 2-phase signals at every node, 200 vehicles, OD 0->99")


def grid64_network(rng):
    """64x64 grid, 10% of road pairs removed (graph kept connected), plus 200 straight arterials."""
    rows = cols = 64
    a, b, length, speed, orient, x, y = grid_roads(rows, cols, rng)
    n = rows * cols
    n_remove = int(round(0.10 * a.size))
    while True:
        drop = rng.choice(a.size, size=n_remove, replace=False)
        keep = np.ones(a.size, bool)
        keep[drop] = False
        if _connected(n, a[keep], b[keep]):
            break
    speed_full = speed.copy()
    a, b, length, speed, orient = a[keep], b[keep], length[keep], speed[keep], orient[keep]
    # arterials: straight links spanning 4..16 cells along a row or a column, length = straight-line
    # distance, speed = 1.5 x the fastest limit among the grid segments they span
    h_speed = speed_full[: rows * (cols - 1)].reshape(rows, cols - 1)
    v_speed = speed_full[rows * (cols - 1):].reshape(rows - 1, cols)
    seen = set()
    art = []
    while len(art) < 200:
        o = int(rng.integers(0, 2))
        line = int(rng.integers(0, 64))
        span = int(rng.integers(4, 17))
        start = int(rng.integers(0, 64 - span))
        if o == 0:
            u, v = line * cols + start, line * cols + start + span
            vmax = int(h_speed[line, start:start + span].max())
        else:
            u, v = start * cols + line, (start + span) * cols + line
            vmax = int(v_speed[start:start + span, line].max())
        if (u, v) in seen:
            continue
        seen.add((u, v))
        art.append((u, v, span * 1000, (3 * vmax) // 2, o))
    art = np.array(art, dtype=np.int64)
    a = np.concatenate([a, art[:, 0]])
    b = np.concatenate([b, art[:, 1]])
    length = np.concatenate([length, art[:, 2]])
    speed = np.concatenate([speed, art[:, 3]])
    orient = np.concatenate([orient, art[:, 4]])
    return csr_from_roads(n, a, b, length, speed, np.full(a.size, 3), orient, x, y)


def grid64(n_queries=16, n_ants=1024, n_iter=200) -> Workload:
    """64x64 perturbed grid (~14.9k directed roads), 2000 Zipf(1.2) vehicles, 16 uniform OD pairs."""
    rng = np.random.Generator(np.random.PCG64(2))
    net = grid64_network(rng)
    sig = two_phase_signals(net, np.ones(net.n_nodes, bool), rng)
    veh = vehicles_zipf(net.n_edges, 2000, 1.2, rng)
    od = uniform_od(net.n_nodes, 16, rng)[:n_queries]
    q = [Query(s, d, n_ants, n_iter, 1.0, 2.0, 0.1, i) for i, (s, d) in enumerate(od)]
    return Workload("grid64", net, sig, veh, q,
                    "64x64 grid minus 10% road pairs plus 200 arterials, 2-phase signals everywhere, "
                    "2000 Zipf(1.2) vehicles, uniform OD pairs")


def thin_lattice(n_nodes, a, b, order, target):
    """Links kept when the links a[i]-b[i] of a connected graph are tried for removal in the order
    ``order`` and each one that is not a bridge of the remaining graph is removed, until ``target``
    links remain.

    Trying links in a fixed order and removing the non-bridges is reverse-delete (Kruskal 1956) with
    the links tried first as the heaviest: run to the end it leaves the minimum spanning tree of those
    weights, and a link it keeps stays a bridge from then on. Stopped early, it has removed the non-tree
    links it reached, so what remains is that tree plus the non-tree links it had not reached yet. Those
    are the ones tried last, i.e. the lightest. That is computed here in O(E log E): a Kruskal spanning
    tree, then the lightest non-tree links until ``target`` links remain.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    m = a.size
    weight = np.empty(m, np.float64)
    weight[np.asarray(order)] = np.arange(m, 0, -1, dtype=np.float64)  # tried first = heaviest
    mst = minimum_spanning_tree(coo_matrix((weight, (a, b)), shape=(n_nodes, n_nodes))).tocoo()
    key = np.minimum(a, b) * n_nodes + np.maximum(a, b)
    tree_key = np.minimum(mst.row, mst.col).astype(np.int64) * n_nodes + np.maximum(mst.row, mst.col)
    in_tree = np.isin(key, tree_key)
    rest = np.flatnonzero(~in_tree)
    rest = rest[np.argsort(weight[rest])]  # lightest (tried last) first
    n_rest = max(0, int(target) - int(in_tree.sum()))
    return np.sort(np.concatenate([np.flatnonzero(in_tree), rest[:n_rest]]))


def geometric_network(n_rows, n_cols, rng, avg_out_degree=2.8, cell_dm=2000, jitter=0.35, lanes=3):
    """Planar road graph on a jittered lattice.

    One point per 200 m cell (jitter +-0.35 cell) with links to its 4 lattice neighbours; random links
    that are not bridges are removed, one at a time, until the average out-degree (directed roads per
    node) is ``avg_out_degree`` (``thin_lattice``). Length = straight-line distance x U[1.0, 1.4];
    speed limits U{30, 50, 70} km/h.
    """
    n = n_rows * n_cols
    gx = (np.arange(n) % n_cols).astype(np.float64)
    gy = (np.arange(n) // n_cols).astype(np.float64)
    x = np.round((gx + rng.uniform(-jitter, jitter, n)) * cell_dm).astype(np.int64)
    y = np.round((gy + rng.uniform(-jitter, jitter, n)) * cell_dm).astype(np.int64)
    ids = np.arange(n).reshape(n_rows, n_cols)
    a = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    b = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    sel = thin_lattice(n, a, b, rng.permutation(a.size), int(round(avg_out_degree * n / 2)))
    a, b = a[sel], b[sel]
    dx = (x[b] - x[a]).astype(np.float64)
    dy = (y[b] - y[a]).astype(np.float64)
    eucl = np.sqrt(dx * dx + dy * dy)
    length = np.maximum(1, np.ceil(eucl * rng.uniform(1.0, 1.4, a.size))).astype(np.int64)
    speed = rng.choice(np.array(SPEEDS_KMH), size=a.size)
    orient = (np.abs(dy) > np.abs(dx)).astype(np.int64)
    return csr_from_roads(n, a, b, length, speed, np.full(a.size, lanes), orient, x, y)


def geo100k(n_queries=512, n_ants=256, n_iter=100) -> Workload:
    """100k-node planar geometric road graph (avg out-degree 2.8), signals at 60% of nodes,
    Poisson(1.0) vehicles per road, OD pairs with BFS hop counts 20..400."""
    rng = np.random.Generator(np.random.PCG64(3))
    net = geometric_network(250, 400, rng)
    sig = two_phase_signals(net, rng.random(net.n_nodes) < 0.6, rng)
    veh = vehicles_poisson(net.n_edges, 1.0, rng)
    od = hop_filtered_od(net, n_queries, 20, 400, rng)
    q = [Query(s, d, n_ants, n_iter, 1.0, 2.0, 0.1, i) for i, (s, d) in enumerate(od)]
    return Workload("geo100k", net, sig, veh, q,
                    "100k-node jittered-lattice planar graph, 60% signalised, Poisson(1) vehicles/road")


def geo1m_serving() -> Workload:
    """1M-node planar road graph (same generator as geo100k, 60% signalised) carrying 5M vehicles placed
    uniformly on its roads; route requests are generated by the serving loop (uniform OD pairs)."""
    rng = np.random.Generator(np.random.PCG64(5))
    net = geometric_network(1000, 1000, rng)
    sig = two_phase_signals(net, rng.random(net.n_nodes) < 0.6, rng)
    veh = vehicles_uniform(net.n_edges, 5_000_000, rng)
    return Workload("geo1m", net, sig, veh, [], "1M-node planar graph, 60% signalised, 5M vehicles")


def city_batch(n_graphs=64, n_min=1000, n_max=200_000, q_lo=8, q_hi=64, ants_lo=128, ants_hi=1024, n_iter=50,
               seed=4) -> list[Workload]:
    """Independent city graphs for one multi-graph launch: node counts log-uniform in [n_min, n_max] (same
    planar generator as geo100k, avg out-degree 2.8, 60% signalised), mean density U[0.5, 3] vehicles per
    road (Poisson), q_lo..q_hi uniform OD queries per graph with ants_lo..ants_hi ants each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for g in range(n_graphs):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        rows = max(2, int(np.sqrt(n)))
        cols = max(2, n // rows)
        net = geometric_network(rows, cols, rng)
        sig = two_phase_signals(net, rng.random(net.n_nodes) < 0.6, rng)
        veh = vehicles_poisson(net.n_edges, float(rng.uniform(0.5, 3.0)), rng)
        nq = int(rng.integers(q_lo, q_hi + 1))
        qs = [Query(s, d, int(rng.integers(ants_lo, ants_hi + 1)), n_iter, 1.0, 2.0, 0.1, 1000 * g + i)
              for i, (s, d) in enumerate(uniform_od(net.n_nodes, nq, rng))]
        out.append(Workload(f"city{g}", net, sig, veh, qs, f"{net.n_nodes}-node planar city graph"))
    return out


def city52(seed=52) -> Workload:
    """52 intersections joined by 64 two-way streets (128 directed roads, 3 lanes): a synthetic network
    of the size of the paper's North-West Delhi map (Sec. 5), whose data is not published. A 4 x 13
    lattice (800 m spacing, +-25 % jitter) keeps 64 of its 87 street segments at random, connected;
    lengths are the straight line x U[1.0, 1.25], speeds U{30,50,70} km/h, 2-phase signals at nodes
    with three or more streets, no background vehicles (the simulated vehicles are the traffic)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols, sp = 4, 13, 8000
    n = rows * cols
    gx, gy = np.meshgrid(np.arange(cols), np.arange(rows))
    x = np.round((gx.ravel() + rng.uniform(-0.25, 0.25, n)) * sp).astype(np.int64)
    y = np.round((gy.ravel() + rng.uniform(-0.25, 0.25, n)) * sp).astype(np.int64)
    pairs = [(r * cols + c, r * cols + c + 1) for r in range(rows) for c in range(cols - 1)]
    pairs += [(r * cols + c, (r + 1) * cols + c) for r in range(rows - 1) for c in range(cols)]
    pa = np.array([p for p, _ in pairs], np.int64)
    pb = np.array([q for _, q in pairs], np.int64)
    while True:
        keep = np.sort(rng.choice(pa.size, size=64, replace=False))
        if _connected(n, pa[keep], pb[keep]):
            break
    a, b = pa[keep], pb[keep]
    dx, dy = np.abs(x[a] - x[b]), np.abs(y[a] - y[b])
    eucl = np.sqrt((dx * dx + dy * dy).astype(np.float64))
    length = np.ceil(eucl * rng.uniform(1.0, 1.25, a.size)).astype(np.int64)
    speed = rng.choice(np.array(SPEEDS_KMH), size=a.size)
    orient = (dy > dx).astype(np.int64)
    net = csr_from_roads(n, a, b, length, speed, np.full(a.size, 3), orient, x, y)
    sig = two_phase_signals(net, np.diff(net.row_ptr.astype(np.int64)) >= 3, rng)
    return Workload("city52", net, sig, np.zeros(net.n_edges, np.uint32), [],
                    "52 intersections, 128 directed roads, 3 lanes, 2-phase signals at 3+-street nodes")


def random_small(n_nodes, n_undirected, rng, signalised_frac=0.0, len_lo=1000, len_hi=5000,
                 spacing_dm=1000) -> tuple[RoadNetwork, SignalTiming]:
    """Small connected random road graph on a sparse lattice layout (for brute-force checks)."""
    side = int(np.ceil(np.sqrt(n_nodes)))
    x = (np.arange(n_nodes) % side) * spacing_dm
    y = (np.arange(n_nodes) // side) * spacing_dm
    while True:
        pairs = set()
        perm = rng.permutation(n_nodes)
        for i in range(1, n_nodes):  # random tree first
            j = int(rng.integers(0, i))
            p, q = int(perm[i]), int(perm[j])
            pairs.add((min(p, q), max(p, q)))
        tries = 0
        while len(pairs) < n_undirected and tries < 10000:
            p, q = (int(v) for v in rng.integers(0, n_nodes, 2))
            tries += 1
            if p != q:
                pairs.add((min(p, q), max(p, q)))
        a = np.array([p for p, _ in pairs], dtype=np.int64)
        b = np.array([q for _, q in pairs], dtype=np.int64)
        if _connected(n_nodes, a, b):
            break
    dx = np.abs(x[a] - x[b])
    dy = np.abs(y[a] - y[b])
    eucl = np.sqrt((dx * dx + dy * dy).astype(np.float64))
    # roads are never shorter than the straight line between their ends
    length = np.maximum(np.ceil(eucl).astype(np.int64), rng.integers(len_lo, len_hi + 1, size=a.size))
    speed = rng.choice(np.array(SPEEDS_KMH), size=a.size)
    orient = (dy > dx).astype(np.int64)
    net = csr_from_roads(n_nodes, a, b, length, speed, np.full(a.size, 3), orient, x, y)
    sig = two_phase_signals(net, rng.random(n_nodes) < signalised_frac, rng)
    return net, sig


WORKLOADS = {"grid10": grid10, "grid64": grid64, "geo100k": geo100k}

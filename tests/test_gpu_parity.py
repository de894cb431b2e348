"""Parity of the sm_103a library (through the C ABI) with the CPU oracle, bit for bit.

Every comparison is exact: routes, travel and wait times, step and success counts, the best
(iteration, ant), per-ant logs, final pheromone tables, road times and phase orders. The tolerance is
zero because both sides use integer arithmetic and identically ordered binary32 operations.
"""
import dataclasses

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
from tests import oracle_pool

pytestmark = pytest.mark.gpu

Q = W.Query


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


# job schedules: the iterative job as one chain, as two and as the default number of concurrent colony
# chains, and the persistent job
FREE = 16  # gmacop.FLAG_NO_LOCKSTEP: sub-warp groups that do not step in lockstep
SCHEDULES = {"chains1": dict(mode=1, branches=1), "chains2": dict(mode=1, branches=2),
             "chains_default": dict(mode=1), "persistent": dict(mode=2),
             "sparse_tau": dict(mode=1, tau_layout=2), "dense_tau": dict(mode=1, tau_layout=1),
             # walks longer than 3 moves finish in the tail kernel (pipelined, one ant per warp)
             "handoff": dict(mode=1, lanes_per_ant=8, flags=FREE, handoff_moves=3)}


def _with_flags(sched, flags):
    kw = dict(SCHEDULES[sched])
    kw["flags"] = kw.get("flags", 0) | flags
    return kw


def _oparams(orc, **kw):
    return orc.Params(**kw)


def _compare(orc, onet, oparams, q, gres, ctx=None, slot=0, log=None):
    o = orc.solve(onet, oparams, q, want_log=log is not None)
    assert gres["status"] == o["status"], (gres, {k: v for k, v in o.items() if k not in ("tau", "log")})
    for k in ("travel_ms", "wait_ms", "ant_steps", "n_success", "route_len"):
        assert gres[k] == o[k], (k, gres[k], o[k])
    if o["status"] == 0:
        assert gres["best_iter"] == o["best_iter"] and gres["best_ant"] == o["best_ant"]
        np.testing.assert_array_equal(gres["route"], o["route"])
    if ctx is not None:
        np.testing.assert_array_equal(ctx.pheromone(slot), o["tau"])
    if log is not None:
        np.testing.assert_array_equal(log, o["log"])
    return o


def test_edge_times_and_phase_order(gm, ctx, orc):
    for wl in (W.grid10(), W.grid64(n_queries=1)):
        ctx.load_workload(wl)
        onet = orc.Net.from_workload(wl)
        prep = orc.prepare(onet, orc.Params(), 0)
        tt, qd = ctx.edge_times()
        np.testing.assert_array_equal(tt, prep["tt"])
        np.testing.assert_array_equal(qd, prep["qd"])
        np.testing.assert_array_equal(ctx.phase_order(), prep["order"])


def test_densities_from_device_memory_and_red_time_round_trip(gm, ctx, orc):
    """Densities written from a device array (gathered into the library's slot order by a kernel) give the
    same road times, queue delays, phase orders and read-back vehicles as the oracle on those vehicles;
    red times written with non-zero entries in every phase slot (also those above a node's phase count,
    which the library keeps in planes the tick does not visit) read back unchanged."""
    torch = pytest.importorskip("torch")
    wl = W.grid64(n_queries=1)
    ctx.load_workload(wl)
    rng = np.random.default_rng(17)
    veh = rng.integers(0, 40, wl.net.n_edges).astype(np.uint32)
    dev = torch.from_numpy(veh.astype(np.int32)).to("cuda:0")
    torch.cuda.synchronize()
    ctx.set_densities_device(dev.data_ptr())
    tt, qd = ctx.edge_times()  # synchronises the context's stream
    del dev
    onet = orc.Net(wl.net, wl.signals, veh)
    prep = orc.prepare(onet, orc.Params(), 0)
    np.testing.assert_array_equal(tt, prep["tt"])
    np.testing.assert_array_equal(qd, prep["qd"])
    np.testing.assert_array_equal(ctx.phase_order(), prep["order"])
    np.testing.assert_array_equal(ctx.densities(), veh)
    red = rng.integers(0, 300_000, size=(wl.net.n_nodes, 8)).astype(np.uint32)
    ctx.set_red_times(red)
    np.testing.assert_array_equal(ctx.red_times(), red)
    np.testing.assert_array_equal(ctx.phase_order(), orc.queue_preempt(orc.Net(wl.net, wl.signals, veh, red)))


def test_phase_order_with_red_times_and_queues(gm, ctx, orc):
    rng = np.random.default_rng(5)
    net, sig = W.random_small(60, 120, rng, signalised_frac=0.7)
    # give some nodes 3-8 phases
    P = np.where(sig.n_phases > 0, rng.integers(2, 9, net.n_nodes), 0).astype(np.uint8)
    green = np.zeros((net.n_nodes, 8), np.uint32)
    for v in range(net.n_nodes):
        if P[v]:
            green[v, : P[v]] = rng.integers(5000, 30000, P[v])
    cycle = green.sum(1).astype(np.uint32)
    offset = (rng.random(net.n_nodes) * np.maximum(cycle, 1)).astype(np.uint32)
    heads = net.col
    ephase = np.where(P[heads] > 0, rng.integers(0, 8, net.n_edges) % np.maximum(P[heads], 1), 0).astype(np.uint8)
    sig = W.SignalTiming(P, cycle, offset, green.ravel(), ephase)
    veh = rng.integers(0, 60, net.n_edges).astype(np.uint32)
    red = rng.choice(np.array([0, 1000, 200000], np.uint32), size=(net.n_nodes, 8))
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    ctx.set_red_times(red)
    onet = orc.Net(net, sig, veh, red)
    np.testing.assert_array_equal(ctx.phase_order(), orc.queue_preempt(onet))
    q = Q(0, net.n_nodes - 1, 64, 10, 1.0, 2.0, 0.1, 9)
    ctx.set_params(flags=gm.FLAG_ANT_LOG)
    r = ctx.solve_batch([q])[0]
    _compare(orc, onet, orc.Params(), q, r, ctx, 0, ctx.ant_log(0))


@pytest.mark.parametrize("mode", [1, 2, "sparse"])
def test_grid10_full_parity(gm, ctx, orc, mode):
    wl = W.grid10()
    ctx.load_workload(wl)
    if mode == "sparse":  # pheromone as a baseline plus the roads with deposits: same tables and routes
        ctx.set_params(flags=gm.FLAG_ANT_LOG, mode=1, tau_layout=gm.TAU_SPARSE)
    else:
        ctx.set_params(flags=gm.FLAG_ANT_LOG, mode=mode)
    q = wl.queries[0]
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(), q, r, ctx, 0, ctx.ant_log(0))


@pytest.mark.parametrize("lanes", [1, 4, 8, 16, 32])
def test_grid10_same_result_for_every_lane_count(gm, ctx, orc, lanes):
    wl = W.grid10(n_ants=48, n_iter=20)
    ctx.load_workload(wl)
    ctx.set_params(lanes_per_ant=lanes)
    r = ctx.solve_batch(wl.queries)[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(), wl.queries[0], r, ctx)


@pytest.mark.parametrize("variant", ["random_tau", "threshold", "t_dep", "max_steps", "hsat", "alpha0beta0",
                                     "alpha2beta3", "no_graph"])
def test_grid10_variants(gm, ctx, orc, variant):
    wl = W.grid10(n_ants=32, n_iter=15)
    ctx.load_workload(wl)
    q = wl.queries[0]
    kw, okw = {}, {}
    if variant == "random_tau":
        kw["flags"] = okw["flags"] = gm.FLAG_RANDOM_TAU
    elif variant == "threshold":
        kw["thr_permille"] = okw["thr_permille"] = 30
    elif variant == "t_dep":
        kw["t_dep_ms"] = okw["t_dep_ms"] = 987_654
    elif variant == "max_steps":
        kw["max_steps"] = okw["max_steps"] = 20
    elif variant == "hsat":
        kw["h_sat_ms"] = okw["h_sat_ms"] = 3100
    elif variant == "alpha0beta0":
        q = Q(q.src, q.dst, q.n_ants, q.n_iter, 0.0, 0.0, 0.25, 3)
    elif variant == "alpha2beta3":
        q = Q(q.src, q.dst, q.n_ants, q.n_iter, 2.0, 3.0, 0.05, 11)
    elif variant == "no_graph":
        kw["flags"] = gm.FLAG_NO_GRAPH
    ctx.set_params(**kw)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(**okw), q, r, ctx)


@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_grid64_batch_parity_reduced(gm, ctx, orc, sched):
    """Four colonies of 256 ants x 20 iterations in one job; each equals its solo oracle solve."""
    wl = W.grid64(n_queries=4, n_ants=256, n_iter=20)
    ctx.load_workload(wl)
    ctx.set_params(**_with_flags(sched, gm.FLAG_ANT_LOG))
    res = ctx.solve_batch(wl.queries)
    onet = orc.Net.from_workload(wl)
    for i, q in enumerate(wl.queries):
        _compare(orc, onet, orc.Params(), q, res[i], ctx, i, ctx.ant_log(i))


@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_ragged_batch_equals_solo(gm, ctx, orc, sched):
    """Different ants, iterations, alpha/beta/rho and seeds per colony, plus src == dst."""
    wl = W.grid64(n_queries=5)
    ctx.load_workload(wl)
    ctx.set_params(**SCHEDULES[sched])
    base = wl.queries
    qs = [Q(base[0].src, base[0].dst, 96, 7, 1.0, 2.0, 0.1, 5),
          Q(base[1].src, base[1].dst, 33, 12, 2.0, 1.0, 0.3, 6),
          Q(base[2].src, base[2].src, 16, 4, 1.0, 2.0, 0.1, 7),
          Q(base[3].src, base[3].dst, 200, 3, 0.0, 3.0, 0.0, 2**40 + 3),
          Q(base[4].src, base[4].dst, 1, 25, 1.0, 2.0, 0.5, 9)]
    res = ctx.solve_batch(qs)
    onet = orc.Net.from_workload(wl)
    for i, q in enumerate(qs):
        _compare(orc, onet, orc.Params(), q, res[i], ctx, i)


@pytest.fixture(scope="module")
def grid64_oracle():
    """The oracle's solves of all 16 benchmark colonies, in spawned processes over the host cores."""
    pool, pending = oracle_pool.start("grid64", range(16))
    try:
        out = pending.get(timeout=3000)
    finally:
        pool.close()
        pool.join()
    return [o for _, o in out]


FULL_SIZE = {"chains": dict(mode=1), "persistent": dict(mode=2),
             "handoff": dict(mode=1, lanes_per_ant=8, flags=FREE, handoff_moves=512)}


@pytest.mark.parametrize("form", list(FULL_SIZE))
def test_grid64_full_size_full_parity(gm, ctx, orc, grid64_oracle, form):
    """The benchmark's job (16 colonies x 1024 ants x 200 iterations, one launch) in the chained form,
    the persistent form and the chained form that hands walks longer than 512 moves to the tail kernel:
    every colony equals the oracle's solve exactly, final pheromone table included."""
    wl = W.grid64()
    ctx.load_workload(wl)
    kw = FULL_SIZE[form]
    mode = kw["mode"]
    ctx.set_params(**kw)  # the benchmark's launch configuration (no timing events)
    ctx.stage(wl.queries)
    ctx.launch()
    res0 = ctx.collect()
    ctx.set_params(**dict(kw, flags=kw.get("flags", 0) | gm.FLAG_KERNEL_TIMING))
    ctx.stage(wl.queries)
    ctx.launch()
    res = ctx.collect()
    for a, b in zip(res0, res):  # events around every kernel change nothing
        assert a["travel_ms"] == b["travel_ms"] and a["ant_steps"] == b["ant_steps"]
        np.testing.assert_array_equal(a["route"], b["route"])
    assert len(grid64_oracle) == len(wl.queries) == 16
    for i, o in enumerate(grid64_oracle):
        oracle_pool.check(res[i], o, ctx.pheromone(i))
    assert all(r["status"] == 0 for r in res)
    # a second launch of the staged batch starts from fresh pheromone: identical results
    ctx.launch()
    res2 = ctx.collect()
    for a, b in zip(res, res2):
        assert a["travel_ms"] == b["travel_ms"] and a["ant_steps"] == b["ant_steps"]
    kt = ctx.kernel_times()  # construction time is summed over concurrent colony chains
    assert kt["construct"] > 0 and kt["job"] > 0
    assert kt["iter_end"] > 0 if mode == 1 else kt["iter_end"] == 0  # the persistent job is one kernel


@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_large_graph_global_visited_sets(gm, ctx, orc, sched):
    """A 40k-node planar graph: visited bitmaps no longer fit in shared memory."""
    rng = np.random.Generator(np.random.PCG64(8))
    net = W.geometric_network(200, 200, rng)
    sig = W.two_phase_signals(net, rng.random(net.n_nodes) < 0.6, rng)
    veh = W.vehicles_poisson(net.n_edges, 1.0, rng)
    wl = W.Workload("geo40k", net, sig, veh)
    od = W.hop_filtered_od(net, 2, 20, 60, rng)
    qs = [Q(s, d, 64, 6, 1.0, 2.0, 0.1, i) for i, (s, d) in enumerate(od)]
    ctx.load_workload(wl)
    ctx.set_params(**SCHEDULES[sched])
    res = ctx.solve_batch(qs)
    onet = orc.Net.from_workload(wl)
    for i, q in enumerate(qs):
        _compare(orc, onet, orc.Params(), q, res[i], ctx, i)


@pytest.mark.parametrize("gseed", range(4))
def test_tiny_signalised_graphs(gm, ctx, orc, gseed):
    rng = np.random.Generator(np.random.PCG64(300 + gseed))
    net, sig = W.random_small(9, 14, rng, signalised_frac=1.0)
    veh = rng.integers(0, 15, net.n_edges).astype(np.uint32)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    q = Q(0, 8, 40, 12, 1.0, 2.0, 0.1, gseed)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net(net, sig, veh), orc.Params(), q, r, ctx)


def test_edge_cases(gm, ctx, orc):
    net, sig, veh = NB.build(4, [(0, 1, 1000, 50), (1, 2, 1000, 50)])  # node 3 unreachable
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    r = ctx.solve(0, 3, 8, 3)
    assert r["status"] == gm.ERR_NO_ROUTE and r["ant_steps"] == 3 * 8 * 4  # 0 -> 1 -> 2, back, back
    r = ctx.solve(2, 2, 8, 3)
    assert r["status"] == 0 and list(r["route"]) == [2] and r["travel_ms"] == 0 and r["ant_steps"] == 0
    r = ctx.solve(0, 2, 8, 3, route_cap=2)
    assert r["status"] == gm.ERR_BUFFER and r["route_len"] == 3
    with pytest.raises(gm.GmpError) as e:
        ctx.solve_batch([Q(0, 2, 8, 3, 8.5, 2.0, 0.1, 0)])
    assert e.value.code == gm.ERR_UNSUPPORTED
    with pytest.raises(gm.GmpError) as e:
        ctx.solve_batch([Q(0, 2, 8, 3, 1.0, float("nan"), 0.1, 0)])
    assert e.value.code == gm.ERR_UNSUPPORTED
    with pytest.raises(gm.GmpError) as e:
        ctx.solve_batch([Q(0, 9, 8, 3, 1.0, 2.0, 0.1, 0)])
    assert e.value.code == gm.ERR_INVALID_ARG
    with pytest.raises(gm.GmpError) as e:
        ctx.solve_batch([])
    assert e.value.code == gm.ERR_INVALID_ARG
    with pytest.raises(gm.GmpError) as e:
        ctx.set_params(t_dep_ms=2**30)
    assert e.value.code == gm.ERR_INVALID_ARG


def test_time_cap_and_step_cap(gm, ctx, orc):
    roads = [(i, i + 1, 10**9, 1) for i in range(17)]
    net, sig, veh = NB.build(18, roads)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    onet = orc.Net(net, sig, veh)
    for dst in (16, 17):
        q = Q(0, dst, 3, 2, 1.0, 2.0, 0.1, 0)
        _compare(orc, onet, orc.Params(), q, ctx.solve_batch([q])[0], ctx)
    ctx.set_params(max_steps=5)
    q = Q(0, 16, 3, 2, 1.0, 2.0, 0.1, 0)
    _compare(orc, onet, orc.Params(max_steps=5), q, ctx.solve_batch([q])[0], ctx)


def test_memory_budget(gm, orc):
    c = gm.Context(0, mem_budget=1 << 20)
    wl = W.grid64(n_queries=1)
    with pytest.raises(gm.GmpError) as e:
        c.load_workload(wl)
        c.solve_batch(wl.queries)
    assert e.value.code == gm.ERR_OOM
    c.close()


@pytest.mark.parametrize("sched", ["lanes1", "lanes4", "lanes8", "lanes16", "lanes32", "persistent"])
def test_directed_graph_with_sinks(gm, ctx, orc, sched):
    """One-way roads and nodes without out-roads: an ant that reaches a sink steps back along its route,
    under every kernel shape, including warps whose every ant sits at a sink in the same step. The
    per-ant logs (status, route length, moves, T, W) agree with the oracle's."""
    rng = np.random.default_rng(17)
    roads = []
    for u in range(45):
        for v in rng.choice(60, size=int(rng.integers(1, 4)), replace=False):
            if v != u:
                roads.append((u, int(v), int(rng.integers(300, 3000)), 50, 3, int(rng.integers(0, 2))))
    sigs = {v: (30_000, int(rng.integers(0, 30_000)), [18_000, 12_000]) for v in range(0, 60, 4)}
    net, sig, veh = NB.build(60, roads, signals=sigs, bidirectional=False)
    veh[:] = rng.integers(0, 20, size=veh.size)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    kw = dict(mode=2, lanes_per_ant=8) if sched == "persistent" else dict(mode=1, lanes_per_ant=int(sched[5:]))
    ctx.set_params(flags=gm.FLAG_ANT_LOG, **kw)
    qs = [Q(s, d, 48, 5, 1.0, 2.0, 0.1, 100 + i) for i, (s, d) in enumerate([(0, 50), (3, 44), (7, 59), (10, 20)])]
    res = ctx.solve_batch(qs)
    onet = orc.Net(net, sig, veh)
    backs = 0
    for i, q in enumerate(qs):
        o = _compare(orc, onet, orc.Params(), q, res[i], ctx, i, ctx.ant_log(i))
        _, length, moves, _, _ = orc.log_fields(o["log"])
        backs += int((moves - length).sum()) // 2
    assert backs > 0  # ants stepped back out of sinks and dead ends


@pytest.mark.parametrize("sched", ["handoff", "lanes8", "lanes4", "persistent"])
def test_roads_from_a_node_to_itself(gm, ctx, orc, sched):
    """A road that leads from a node back to itself is never a way on (the node is visited once the ant
    stands on it). Every kernel shape, the hand-off schedule included, agrees with the oracle on a graph
    where a third of the nodes carry such a road."""
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
    assert int(np.diff(net.row_ptr).max()) <= 8
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    if sched == "handoff":
        kw = dict(mode=1, lanes_per_ant=8, flags=FREE, handoff_moves=3)
    elif sched == "persistent":
        kw = dict(mode=2, lanes_per_ant=8)
    else:
        kw = dict(mode=1, lanes_per_ant=int(sched[5:]))
    ctx.set_params(**kw)
    qs = [Q(s, d, 40, 6, 1.0, 2.0, 0.1, 300 + i) for i, (s, d) in enumerate([(0, 47), (3, 30), (9, 21)])]
    res = ctx.solve_batch(qs)
    onet = orc.Net(net, sig, veh)
    for i, q in enumerate(qs):
        _compare(orc, onet, orc.Params(), q, res[i], ctx, i)


def test_sparse_layout_refusals(gm, ctx):
    ctx.load_workload(W.grid10())
    q = W.grid10().queries[0]
    for kw in (dict(mode=2, tau_layout=2), dict(mode=1, tau_layout=2, flags=gm.FLAG_RANDOM_TAU)):
        ctx.set_params(**kw)
        with pytest.raises(gm.GmpError) as ei:
            ctx.solve_batch([q])
        assert ei.value.code == gm.ERR_UNSUPPORTED
    with pytest.raises(gm.GmpError) as ei:
        ctx.set_params(tau_layout=3)
    assert ei.value.code == gm.ERR_INVALID_ARG


@pytest.mark.parametrize("deg", [20, 100])
def test_high_degree_hub(gm, ctx, orc, deg):
    """A hub with `deg` one-way roads out (several candidate slots per lane, up to the 128-road limit of
    32 lanes x 4 slots), each spoke leading to the destination."""
    roads = [(0, 1 + i, 1000 + 37 * i, 50, 3, 0) for i in range(deg)]
    roads += [(1 + i, deg + 1, 2000 + 91 * (deg - i), 50, 3, 0) for i in range(deg)]
    net, sig, veh = NB.build(deg + 2, roads, bidirectional=False)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    q = Q(0, deg + 1, 64, 8, 1.0, 2.0, 0.1, deg)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net(net, sig, veh), orc.Params(), q, r, ctx, 0)


def test_degree_above_limit_is_refused(gm, ctx):
    roads = [(0, 1 + i, 1000, 50, 3, 0) for i in range(130)] + [(1, 131, 1000, 50, 3, 0)]
    net, sig, veh = NB.build(132, roads, bidirectional=False)
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    with pytest.raises(gm.GmpError) as ei:
        ctx.solve_batch([Q(0, 131, 8, 2, 1.0, 2.0, 0.1, 0)])
    assert ei.value.code == gm.ERR_UNSUPPORTED


def test_consecutive_jobs_on_one_context(gm, ctx, orc):
    """Iterative jobs do not clear the deposit accumulators at init (each job leaves them zero); a context
    that runs jobs of growing and shrinking size, switching between the persistent job and both pheromone
    layouts, must still match the oracle colony for colony."""
    wl = W.grid64(n_queries=6, n_ants=64, n_iter=6)
    ctx.load_workload(wl)
    onet = orc.Net.from_workload(wl)
    plan = [(dict(mode=1), [0, 1, 2]), (dict(mode=1), [0, 1, 2, 3, 4, 5]), (dict(mode=2), [3, 4]),
            (dict(mode=1, tau_layout=2), [5, 4, 3, 2]), (dict(mode=1, tau_layout=1), [1]),
            (dict(mode=1), [2, 0, 5, 1, 4])]
    for n, (kw, idx) in enumerate(plan):
        qs = [dataclasses.replace(wl.queries[i], seed=100 * n + i) for i in idx]
        ctx.set_params(**kw)
        res = ctx.solve_batch(qs)
        for j, q in enumerate(qs):
            _compare(orc, onet, orc.Params(), q, res[j], ctx, j)


@pytest.mark.parametrize("sched", ["chains_default", "chains1", "persistent"])
def test_queue_update_fast_and_general_paths(gm, ctx, orc, sched):
    """Intersections with one or two phases take the iteration end's small path, the others a general pass
    of their own: a graph mixing 0-8 phases, heavy queues (some over 3/4 of capacity) and long red times
    (some starved) must keep the oracle's phase orders through a multi-iteration job."""
    rng = np.random.default_rng(31)
    net, sig = W.random_small(200, 420, rng, signalised_frac=0.8)
    P = np.where(sig.n_phases > 0, rng.choice([1, 2, 2, 2, 3, 5, 8], net.n_nodes), 0).astype(np.uint8)
    green = np.zeros((net.n_nodes, 8), np.uint32)
    for v in range(net.n_nodes):
        if P[v]:
            green[v, : P[v]] = rng.integers(4000, 30000, P[v])
    cycle = green.sum(1).astype(np.uint32)
    offset = (rng.random(net.n_nodes) * np.maximum(cycle, 1)).astype(np.uint32)
    ephase = np.where(P[net.col] > 0, rng.integers(0, 8, net.n_edges) % np.maximum(P[net.col], 1), 0).astype(np.uint8)
    sig = W.SignalTiming(P, cycle, offset, green.ravel(), ephase)
    veh = rng.integers(0, 120, net.n_edges).astype(np.uint32)
    red = rng.choice(np.array([0, 3000, 90000, 400000], np.uint32), size=(net.n_nodes, 8))
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    ctx.set_red_times(red)
    ctx.set_params(**SCHEDULES[sched])
    onet = orc.Net(net, sig, veh, red)
    want = orc.queue_preempt(onet)
    np.testing.assert_array_equal(ctx.phase_order(), want)
    qs = [Q(int(s), int(d), 24, 7, 1.0, 2.0, 0.1, 60 + i) for i, (s, d) in enumerate(W.uniform_od(net.n_nodes, 5, rng))]
    res = ctx.solve_batch(qs)
    for i, q in enumerate(qs):
        _compare(orc, onet, orc.Params(), q, res[i], ctx, i)
    np.testing.assert_array_equal(ctx.phase_order(), want)
    tt, qd = ctx.edge_times()
    prep = orc.prepare(onet, orc.Params(), 0)
    np.testing.assert_array_equal(tt, prep["tt"])

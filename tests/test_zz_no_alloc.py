"""gmp_solve_static, the colony solve that allocates no device memory, against gmp_solve.

Some callers cannot call cudaMalloc while they solve: a loop that must never wait on the device
allocator, a memory pool or quota that is already used up, or a framework that owns every allocation.
gmp_solve_static serves them by keeping all of its temporaries in one fixed device array inside the
library and writing its result into device buffers the caller already holds. These tests check that
it returns exactly what gmp_solve returns, on consecutive calls that reuse the array the previous call
left behind, and that it refuses work that does not fit the array or the caller's route buffer.
"""
import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROW = np.dtype([("travel_ms", "<u8"), ("wait_ms", "<u8"), ("ant_steps", "<u8"), ("n_success", "<u8"),
                ("route_len", "<u4"), ("best_iter", "<u4"), ("best_ant", "<u4"), ("status", "<i4")])


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


def _static(gm, ctx, q, route_cap):
    import torch

    row = torch.zeros(ROW.itemsize, dtype=torch.uint8, device="cuda")
    route = torch.zeros(route_cap, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    ctx.solve_static(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed, row.data_ptr(),
                     route.data_ptr(), route_cap)
    torch.cuda.synchronize()
    r = np.frombuffer(row.cpu().numpy().tobytes(), dtype=ROW)[0]
    return r, route.cpu().numpy().astype(np.uint32)


def test_static_solve_equals_solve_on_consecutive_calls(gm):
    wl = W.grid10()
    ctx = gm.Context(0)
    ctx.load_workload(wl)
    q0 = wl.queries[0]
    q1 = W.Query(7, 93, 40, 30, 1.0, 3.0, 0.2, 11)
    cap = wl.net.n_nodes  # max_steps + 1 for this graph
    for q in (q0, q1, q0):
        ref = ctx.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed)
        row, route = _static(gm, ctx, q, cap)
        assert int(row["status"]) == ref["status"] == gm.OK
        for k in ("travel_ms", "wait_ms", "ant_steps", "n_success", "route_len", "best_iter", "best_ant"):
            assert int(row[k]) == ref[k], (k, int(row[k]), ref[k])
        np.testing.assert_array_equal(route[: ref["route_len"]], ref["route"])
    ctx.close()


def _multi_phase_workload(seed):
    """A 200-node graph whose intersections have 0-8 phases (some over two, so the general queue pass
    runs), heavy queues and long red times."""
    rng = np.random.default_rng(seed)
    net, sig = W.random_small(200, 420, rng, signalised_frac=0.8)
    P = np.where(sig.n_phases > 0, rng.choice([1, 2, 3, 5, 8], net.n_nodes), 0).astype(np.uint8)
    green = np.zeros((net.n_nodes, 8), np.uint32)
    for v in range(net.n_nodes):
        if P[v]:
            green[v, : P[v]] = rng.integers(4000, 30000, P[v])
    cycle = green.sum(1).astype(np.uint32)
    offset = (rng.random(net.n_nodes) * np.maximum(cycle, 1)).astype(np.uint32)
    ephase = np.where(P[net.col] > 0, rng.integers(0, 8, net.n_edges) % np.maximum(P[net.col], 1), 0)
    sig = W.SignalTiming(P, cycle, offset, green.ravel(), ephase.astype(np.uint8))
    veh = rng.integers(0, 120, net.n_edges).astype(np.uint32)
    red = rng.choice(np.array([0, 3000, 90000, 400000], np.uint32), size=(net.n_nodes, 8))
    return W.Workload("phases", net, sig, veh), red, [W.Query(int(s), int(d), 24, 7, 1.0, 2.0, 0.1, 60 + i)
                                                      for i, (s, d) in enumerate(W.uniform_od(net.n_nodes, 3, rng))]


def _geo40k():
    """A 40k-node planar graph: the visited sets no longer fit in shared memory, so the solve carves
    them out of the array as well."""
    rng = np.random.Generator(np.random.PCG64(8))
    net = W.geometric_network(200, 200, rng)
    sig = W.two_phase_signals(net, rng.random(net.n_nodes) < 0.6, rng)
    veh = W.vehicles_poisson(net.n_edges, 1.0, rng)
    od = W.hop_filtered_od(net, 2, 20, 60, rng)
    return W.Workload("geo40k", net, sig, veh), [W.Query(s, d, 64, 4, 1.0, 2.0, 0.1, i) for i, (s, d) in enumerate(od)]


def _same(gm, ctx, q, cap):
    ref = ctx.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed)
    row, route = _static(gm, ctx, q, cap)
    assert int(row["status"]) == ref["status"]
    for k in ("travel_ms", "wait_ms", "ant_steps", "n_success", "route_len", "best_iter", "best_ant"):
        assert int(row[k]) == ref[k], (k, int(row[k]), ref[k])
    if ref["status"] == gm.OK:
        np.testing.assert_array_equal(route[: ref["route_len"]], ref["route"])


def test_static_solve_with_many_phase_signals(gm):
    """Intersections with more than two phases take a queue pass of their own every iteration, in the
    static solve as in the ordinary one."""
    wl, red, qs = _multi_phase_workload(31)
    ctx = gm.Context(0)
    ctx.load_workload(wl)
    ctx.set_red_times(red)
    for q in qs + qs[:1]:  # the last call reuses the array the others left behind
        _same(gm, ctx, q, wl.net.n_nodes)
    ctx.close()


def test_static_solve_with_visited_sets_in_the_array(gm):
    wl, qs = _geo40k()
    ctx = gm.Context(0)
    ctx.load_workload(wl)
    cap = min(wl.net.n_nodes - 1, 4096) + 1
    for q in qs + qs[:1]:
        _same(gm, ctx, q, cap)
    ctx.close()


def test_static_solve_refuses_what_does_not_fit(gm):
    wl = W.grid10()
    ctx = gm.Context(0)
    ctx.load_workload(wl)
    q = wl.queries[0]
    with pytest.raises(gm.GmpError) as e:  # route buffer shorter than max_steps + 1
        _static(gm, ctx, q, 10)
    assert e.value.code == gm.ERR_BUFFER
    big = W.Query(q.src, q.dst, 100_000, 2, 1.0, 2.0, 0.1, 0)  # 100k ants x 99 steps x 4 B > 32 MiB
    with pytest.raises(gm.GmpError) as e:
        _static(gm, ctx, big, wl.net.n_nodes)
    assert e.value.code == gm.ERR_BUFFER
    ctx.close()

"""Serving: continuous batching over slot contexts with traffic ticks between jobs.

Each served result must equal the same request solved alone on a context whose traffic state went
through the same ticks (and departing at the same clock), bit for bit; a sample is also checked against
the oracle's tick chain and colony. The slots share one road graph and traffic state; admission follows
the server's memory budget."""
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


def _mixed_requests(n_nodes, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        s = int(rng.integers(n_nodes))
        d = int(rng.integers(n_nodes - 1))
        d += d >= s
        out.append(W.Query(s, d, int(rng.choice([16, 48, 64])), int(rng.choice([3, 5, 8])), 1.0, 2.0, 0.1,
                           1000 + 7 * i))
    return out


def _same(a, b):
    for k in ("status", "travel_ms", "wait_ms", "ant_steps", "n_success", "best_iter", "best_ant", "route_len"):
        assert a[k] == b[k], (k, a[k], b[k])
    np.testing.assert_array_equal(a["route"], b["route"])


def test_served_equals_alone_and_oracle(gm, orc):
    from paper_2010_14244_gb300 import serving

    wl = W.grid10()
    srv, slots = serving.make_server(wl, n_slots=3, max_batch=6, max_ants=64, max_iter=8)
    reqs = _mixed_requests(wl.net.n_nodes, 30, seed=3)
    ticks = [(0, 1000), (1000, 2500), (3500, 700)]
    done = []
    try:
        # waves: submit some, pump (jobs start), tick between waves while jobs are still on the GPU
        waves = [reqs[0:9], reqs[9:14], reqs[14:25], reqs[25:30]]
        for w, wave in enumerate(waves):
            for i, q in enumerate(wave):
                srv.submit(q, reqs.index(q))
                if i % 3 == 2:
                    srv.pump()
            srv.pump()
            done += srv.take()
            if w < len(ticks):
                srv.tick(*ticks[w])
        for _ in range(200000):
            st = srv.pump()
            done += srv.take()
            if st["queued"] == 0 and st["in_flight"] == 0 and st["done_waiting"] == 0:
                break
        assert len(done) == len(reqs) and sorted(r["tag"] for r in done) == list(range(len(reqs)))
        assert max(r["batch_size"] for r in done) > 1
        assert len({r["slot"] for r in done}) > 1
        clocks = sorted({r["clock_ms"] for r in done})
        assert len(clocks) > 1
    finally:
        srv.close()
        for c in slots:
            c.close()
    # the same requests alone, on a context replaying the ticks
    ref = gm.Context(0)
    try:
        ref.load_workload(wl)
        by_clock = {}
        for r in done:
            by_clock.setdefault(r["clock_ms"], []).append(r)
        clock = 0
        pending = list(ticks)
        while True:
            for r in by_clock.pop(clock, []):
                q = reqs[r["tag"]]
                ref.set_params(t_dep_ms=clock)
                alone = ref.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed)
                _same(r, alone)
            if not pending:
                break
            t, dt = pending.pop(0)
            ref.tick(t, dt)
            clock = t + dt
        assert not by_clock
    finally:
        ref.close()
    # a sample against the oracle: its own tick chain, then the colony departing at that clock
    veh = wl.vehicles.copy()
    red = np.zeros((wl.net.n_nodes, 8), np.uint32)
    order = orc.queue_preempt(orc.Net(wl.net, wl.signals, veh, red))
    states = {0: (veh, red)}
    for t, dt in ticks:
        veh, red, order = orc.tick(orc.Net(wl.net, wl.signals, veh, red), orc.Params(), t, dt, order)
        states[t + dt] = (veh, red)
    for r in done[::5]:
        v, rd = states[r["clock_ms"]]
        o = orc.solve(orc.Net(wl.net, wl.signals, v, rd), orc.Params(t_dep_ms=r["clock_ms"]), reqs[r["tag"]],
                      want_tau=False)
        assert r["status"] == o["status"] and r["travel_ms"] == o["travel_ms"] and r["wait_ms"] == o["wait_ms"]
        if o["status"] == 0:
            np.testing.assert_array_equal(r["route"], o["route"])


def test_admission_follows_memory_budget(gm):
    """The server's budget bounds the memory the slots' workspaces hold together: with room for a few
    requests' tables and routes, jobs are cut down to what fits next to the other slot's, no pump ever
    finds the slots above the budget, and every request still completes."""
    from paper_2010_14244_gb300 import serving

    wl = W.grid64(n_queries=1)
    budget = 64 << 20
    srv, slots = serving.make_server(wl, n_slots=2, max_batch=512, max_ants=256, max_iter=10, mem_budget=budget)
    try:
        assert srv.memory() == (0, budget)
        reqs = _mixed_requests(wl.net.n_nodes, 200, seed=4)
        for i, q in enumerate(reqs):
            srv.submit(dataclasses.replace(q, n_iter=2), i)
        done, peak = [], 0
        for _ in range(200000):
            st = srv.pump()
            done += srv.take()
            peak = max(peak, srv.memory()[0])
            assert srv.memory()[0] <= budget
            if st["queued"] == 0 and st["in_flight"] == 0 and st["done_waiting"] == 0:
                break
        assert len(done) == len(reqs) and all(r["status"] == gm.OK for r in done)
        assert 1 <= max(r["batch_size"] for r in done) < 200
        assert peak > budget // 4
    finally:
        srv.close()
        for c in slots:
            c.close()


def test_views_share_one_graph(gm, orc):
    """gmp_share_graph: a view reads its owner's road graph and traffic state in place and solves exactly
    like it; a view with a traffic state of its own ticks without touching the owner's; what a view may not
    change is refused; an owner with views cannot load another graph."""
    wl = W.grid10()
    owner, view, twin, ref = gm.Context(0), gm.Context(0), gm.Context(0), gm.Context(0)
    try:
        owner.load_workload(wl)
        ref.load_workload(wl)
        view.share_graph(owner)
        twin.share_graph(owner, own_state=True)
        q = wl.queries[0]
        base = owner.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed)
        for c in (view, twin):
            _same(c.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed), base)
        for call in (lambda: view.set_densities(wl.vehicles), lambda: view.tick(0, 1000),
                     lambda: view.set_params(h_sat_ms=2500), lambda: twin.set_signals(wl.signals),
                     lambda: owner.load_workload(wl)):
            with pytest.raises(gm.GmpError) as e:
                call()
            assert e.value.code == gm.ERR_STATE
        # the twin's own traffic state moves on alone: it equals a separate context ticked the same way
        twin.tick(0, 1000)
        ref.tick(0, 1000)
        np.testing.assert_array_equal(twin.densities(), ref.densities())
        np.testing.assert_array_equal(twin.phase_order(), ref.phase_order())
        twin.set_params(t_dep_ms=1000)
        ref.set_params(t_dep_ms=1000)
        _same(twin.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed),
              ref.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed))
        np.testing.assert_array_equal(owner.densities(), wl.vehicles)
        np.testing.assert_array_equal(view.densities(), wl.vehicles)  # read through the owner's tables
        np.testing.assert_array_equal(twin.red_times(), ref.red_times())
        _same(view.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed), base)
    finally:
        for c in (view, twin, owner, ref):
            c.close()


def test_submit_refuses_bad_requests(gm):
    from paper_2010_14244_gb300 import serving

    wl = W.grid10()
    srv, slots = serving.make_server(wl, n_slots=1, max_batch=4, max_ants=32, max_iter=4)
    try:
        with pytest.raises(gm.GmpError) as ei:
            srv.submit(W.Query(0, 99, 64, 2, 1.0, 2.0, 0.1, 1), 0)
        assert ei.value.code == gm.ERR_INVALID_ARG
        with pytest.raises(gm.GmpError) as ei:
            srv.submit(W.Query(0, 100, 8, 2, 1.0, 2.0, 0.1, 1), 1)
        assert ei.value.code == gm.ERR_INVALID_ARG
        with pytest.raises(gm.GmpError) as ei:
            srv.submit(W.Query(0, 9, 8, 2, 9.0, 2.0, 0.1, 1), 2)
        assert ei.value.code == gm.ERR_UNSUPPORTED
        with pytest.raises(gm.GmpError) as ei:
            srv.tick((1 << 30) - 10, 100)
        assert ei.value.code == gm.ERR_INVALID_ARG
        assert srv.pump()["rejected"] == 3
    finally:
        srv.close()
        for c in slots:
            c.close()


def test_poisson_loop_reports_latency(gm):
    from paper_2010_14244_gb300 import serving

    wl = W.grid64(n_queries=1)
    srv, slots = serving.make_server(wl, n_slots=4, max_batch=64, max_ants=128, max_iter=10)
    try:
        rep = serving.run_poisson(srv, serving.uniform_requests(wl.net.n_nodes, 128, 10, seed=1), rate_per_s=400,
                                  duration_s=1.5, warmup_s=0.3, tick_ms=500)
        s = rep.summary()
        assert rep.completed == rep.submitted > 100
        assert s["ticks"] >= 2 and s["p50_ms"] <= s["p99_ms"]
        assert s["queries_per_s"] > 100
    finally:
        srv.close()
        for c in slots:
            c.close()


def test_served_variants_equal_alone(gm):
    """Slots running the exact heuristic with the paper-literal rules serve requests with integer and
    non-integer exponents; each result equals the same request solved alone with the same options."""
    from paper_2010_14244_gb300 import serving

    wl = W.grid10()
    opts = dict(flags=gm.FLAG_EXACT_H | gm.FLAG_PAPER_LITERAL)
    srv, slots = serving.make_server(wl, n_slots=2, max_batch=5, max_ants=64, max_iter=8, params=opts)
    reqs = _mixed_requests(wl.net.n_nodes, 14, seed=21)
    reqs = [dataclasses.replace(q, alpha=q.alpha + (0.5 if i % 2 else 0.0)) for i, q in enumerate(reqs)]
    done = []
    try:
        for i, q in enumerate(reqs):
            srv.submit(q, i)
            if i % 4 == 3:
                srv.pump()
        for _ in range(200000):
            st = srv.pump()
            done += srv.take()
            if st["queued"] == 0 and st["in_flight"] == 0 and st["done_waiting"] == 0:
                break
    finally:
        srv.close()
        for c in slots:
            c.close()
    assert sorted(r["tag"] for r in done) == list(range(len(reqs)))
    ref = gm.Context(0)
    try:
        ref.load_workload(wl)
        ref.set_params(**opts)
        for r in done:
            q = reqs[r["tag"]]
            _same(r, ref.solve(q.src, q.dst, q.n_ants, q.n_iter, q.alpha, q.beta, q.rho, q.seed))
    finally:
        ref.close()

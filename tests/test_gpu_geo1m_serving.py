"""Serving on the 1M-node graph (5M vehicles, the full-size serving network): a short continuously
batched run with 1 s traffic ticks between waves of requests, on two slots. A deterministic sample (every
8th request) is re-solved by the oracle against the traffic state the request saw, obtained by the
oracle's own chain of ticks: status, times, ant-steps, successes and the route must agree bit for bit."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TICKS = [(0, 1000), (1000, 1000)]
N_REQ = 48


def _requests(n_nodes):
    from paper_2010_14244_gb300 import serving

    make = serving.uniform_requests(n_nodes, 128, 30, seed=17)
    return [make(i) for i in range(N_REQ)]


def _oracle_sample(items):
    """items: [(tag, clock_ms)]; replays the ticks on the oracle and solves each sampled request."""
    from oracle import oracle as orc

    wl = W.geo1m_serving()
    reqs = _requests(wl.net.n_nodes)
    veh, red = wl.vehicles.copy(), np.zeros((wl.net.n_nodes, 8), np.uint32)
    order = orc.queue_preempt(orc.Net(wl.net, wl.signals, veh, red))
    states = {0: (veh, red)}
    for t, dt in TICKS:
        veh, red, order = orc.tick(orc.Net(wl.net, wl.signals, veh, red), orc.Params(), t, dt, order)
        states[t + dt] = (veh, red)
    out = []
    for tag, clock in items:
        v, r = states[clock]
        o = orc.solve(orc.Net(wl.net, wl.signals, v, r), orc.Params(t_dep_ms=clock), reqs[tag], want_tau=False)
        out.append({k: o[k] for k in ("status", "travel_ms", "wait_ms", "ant_steps", "n_success")} |
                   {"route": o.get("route")})
    return out


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


def test_geo1m_served_sample_matches_oracle(gm):
    from paper_2010_14244_gb300 import serving

    wl = W.geo1m_serving()
    reqs = _requests(wl.net.n_nodes)
    srv, slots = serving.make_server(wl, n_slots=2, max_batch=12, max_ants=128, max_iter=30)
    done = []
    try:
        waves = [reqs[0:16], reqs[16:32], reqs[32:48]]
        for w, wave in enumerate(waves):
            for q in wave:
                srv.submit(q, reqs.index(q))
            for _ in range(200000):  # the wave completes before the traffic moves on
                st = srv.pump()
                done += srv.take()
                if st["queued"] == 0 and st["in_flight"] == 0 and st["done_waiting"] == 0:
                    break
            if w < len(TICKS):
                srv.tick(*TICKS[w])
    finally:
        srv.close()
        for c in slots:
            c.close()
    assert sorted(r["tag"] for r in done) == list(range(N_REQ))
    by_tag = {r["tag"]: r for r in done}
    assert {r["clock_ms"] for r in done} == {0, 1000, 2000}
    sample = [(tag, int(by_tag[tag]["clock_ms"])) for tag in range(0, N_REQ, 8)]
    # the oracle runs in a process of its own (spawned: it inherits no CUDA state)
    with mp.get_context("spawn").Pool(1) as pool:
        oracle = pool.apply(_oracle_sample, (sample,))
    for (tag, _), o in zip(sample, oracle):
        r = by_tag[tag]
        for k in ("status", "travel_ms", "wait_ms", "ant_steps", "n_success"):
            assert r[k] == o[k], (tag, k, r[k], o[k])
        if o["status"] == 0:
            np.testing.assert_array_equal(r["route"], o["route"])

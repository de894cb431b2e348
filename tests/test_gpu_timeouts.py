"""Bounded device waits run out into GMP_ERR_TIMEOUT and leave the context usable.

Two parts of the library wait on the device: the persistent job, whose groups poll their colony's state
word until the colony moves to its next phase, and the exact heuristic's relaxation, which runs level
after level until its frontiers are empty. Each has a bound (a number of polls, a number of levels) after
which it stops, records an error word and returns; the host then reports GMP_ERR_TIMEOUT. The bounds are
parameters, so a test can make them tiny and watch an ordinary job run out: no trap, no fault, no wait
without a limit. The same context must then solve the same colony with the default bounds and agree with
the oracle bit for bit.
"""
import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


def _same_as_oracle(orc, wl, params, res):
    o = orc.solve(orc.Net.from_workload(wl), params, wl.queries[0], want_tau=False)
    assert res["status"] == o["status"] == 0
    for k in ("travel_ms", "wait_ms", "ant_steps", "n_success", "best_iter", "best_ant"):
        assert res[k] == o[k], (k, res[k], o[k])
    np.testing.assert_array_equal(res["route"], o["route"])


def test_persistent_job_wait_runs_out(gm, orc):
    """One poll allowed: groups without an ant wait for the iteration end at once and give up on their
    second poll, long before the ants' walks are over."""
    wl = W.grid10()
    ctx = gm.Context(0)
    try:
        ctx.load_workload(wl)
        ctx.set_params(mode=gm.MODE_PERSISTENT, lanes_per_ant=8, poll_limit=1)
        with pytest.raises(gm.GmpError) as e:
            ctx.solve_batch(wl.queries[:1])
        assert e.value.code == gm.ERR_TIMEOUT
        ctx.set_params(mode=gm.MODE_PERSISTENT, lanes_per_ant=8)
        _same_as_oracle(orc, wl, orc.Params(), ctx.solve_batch(wl.queries[:1])[0])
    finally:
        ctx.close()


def test_exact_heuristic_level_bound_runs_out(gm, orc):
    """One relaxation level allowed: the pass from the destination stops long before it reaches the
    source (18 roads away on the 10 x 10 grid)."""
    wl = W.grid10()
    ctx = gm.Context(0)
    try:
        ctx.load_workload(wl)
        ctx.set_params(flags=gm.FLAG_EXACT_H, level_limit=1)
        with pytest.raises(gm.GmpError) as e:
            ctx.solve_batch(wl.queries[:1])
        assert e.value.code == gm.ERR_TIMEOUT
        ctx.set_params(flags=gm.FLAG_EXACT_H)
        _same_as_oracle(orc, wl, orc.Params(flags=orc.FLAG_EXACT_H), ctx.solve_batch(wl.queries[:1])[0])
    finally:
        ctx.close()

"""gmp_bind_workspace: a context that carves its device memory from a caller-owned tensor computes what an
ordinary context computes, through batches that grow and shrink (allocations freed and carved again),
refuses what does not fit or is not device memory, and never frees the caller's memory."""
import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


def _same(a, b):
    for k in ("status", "travel_ms", "wait_ms", "ant_steps", "n_success", "best_iter", "best_ant", "route_len"):
        assert a[k] == b[k], (k, a[k], b[k])
    np.testing.assert_array_equal(a["route"], b["route"])


def test_bound_workspace_equals_ordinary_context(gm):
    import torch

    arena = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    wl = W.grid64(n_queries=6, n_ants=128, n_iter=8)
    ref, ctx = gm.Context(0), gm.Context(0)
    try:
        ctx.bind_workspace(arena.data_ptr(), arena.numel())
        ctx.load_workload(wl)
        ref.load_workload(wl)
        for idx, flags in [([0, 1], 0), (list(range(6)), 0), ([2, 3, 4], gm.FLAG_EXACT_H), (list(range(6)), 0),
                           ([5], gm.FLAG_PAPER_LITERAL)]:
            batch = [wl.queries[i] for i in idx]
            for c in (ctx, ref):
                c.set_params(flags=flags)
            got, want = ctx.solve_batch(batch), ref.solve_batch(batch)
            for i, (a, b) in enumerate(zip(got, want)):
                _same(a, b)
                np.testing.assert_array_equal(ctx.pheromone(i), ref.pheromone(i))
    finally:
        ctx.close()
        ref.close()
    arena.fill_(7)  # still the caller's memory after the context is gone
    torch.cuda.synchronize()
    assert int(arena[12345]) == 7


def test_bound_workspace_refusals(gm):
    import torch

    small = torch.empty(256 << 10, dtype=torch.uint8, device="cuda")
    ctx = gm.Context(0)
    try:
        ctx.bind_workspace(small.data_ptr(), small.numel())
        with pytest.raises(gm.GmpError) as e:
            ctx.load_workload(W.grid64(n_queries=1))  # ~1.2 MB of graph and traffic state
        assert e.value.code == gm.ERR_OOM
    finally:
        ctx.close()
    ctx = gm.Context(0)
    try:
        with pytest.raises(gm.GmpError) as e:
            ctx.bind_workspace(small.data_ptr() + 4, 4096)  # not 256-byte aligned
        assert e.value.code == gm.ERR_INVALID_ARG
        host = np.zeros(1 << 16, np.uint8)
        with pytest.raises(gm.GmpError) as e:
            ctx.bind_workspace(host.ctypes.data, host.nbytes)  # host memory
        assert e.value.code == gm.ERR_INVALID_ARG
        ctx.load_workload(W.grid10())
        with pytest.raises(gm.GmpError) as e:
            ctx.bind_workspace(small.data_ptr(), small.numel())  # the context already holds device memory
        assert e.value.code == gm.ERR_STATE
        assert ctx.solve(0, 99, 16, 3)["status"] in (gm.OK, gm.ERR_NO_ROUTE)
    finally:
        ctx.close()

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

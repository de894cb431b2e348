"""Parity of colonies with non-integer alpha / beta (the 2^L score), GPU against the oracle bit for bit,
through the C ABI: every schedule and kernel shape, the paper-literal flags, and jobs that mix integer
and non-integer colonies in the same warps."""
import dataclasses

import pytest

from paper_2010_14244_gb300 import workloads as W
from tests.test_gpu_parity import SCHEDULES, _compare, _with_flags

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


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("ab", [(1.5, 2.5), (0.5, 1.0), (2.0, 0.75), (0.0, 3.25)])
def test_grid10_fractional_exponents(gm, ctx, orc, ab, sched):
    wl = W.grid10(n_ants=32, n_iter=12)
    ctx.load_workload(wl)
    ctx.set_params(**_with_flags(sched, gm.FLAG_ANT_LOG))
    q = Q(wl.queries[0].src, wl.queries[0].dst, 32, 12, ab[0], ab[1], 0.15, 31)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(), q, r, ctx, 0, ctx.ant_log(0))


@pytest.mark.parametrize("lanes", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("lockstep", [True, False])
def test_grid10_fractional_every_kernel_shape(gm, ctx, orc, lanes, lockstep):
    wl = W.grid10(n_ants=48, n_iter=10)
    ctx.load_workload(wl)
    ctx.set_params(lanes_per_ant=lanes, flags=0 if lockstep else gm.FLAG_NO_LOCKSTEP)
    q = Q(wl.queries[0].src, wl.queries[0].dst, 48, 10, 1.25, 2.5, 0.1, 5)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(), q, r, ctx)


def test_fractional_paper_literal(gm, ctx, orc):
    wl = W.grid10(n_ants=32, n_iter=15)
    ctx.load_workload(wl)
    ctx.set_params(flags=gm.FLAG_PAPER_LITERAL)
    q = Q(wl.queries[0].src, wl.queries[0].dst, 32, 15, 2.5, 1.5, 0.2, 8)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(flags=gm.FLAG_PAPER_LITERAL), q, r, ctx)


@pytest.mark.parametrize("sched", ["chains_default", "chains1", "persistent", "sparse_tau"])
def test_mixed_integer_and_fractional_colonies(gm, ctx, orc, sched):
    """Colonies of 6 to 40 ants share warps across colony boundaries; integer and non-integer colonies
    alternate, each equal to its own oracle solve."""
    wl = W.grid64(n_queries=8, n_ants=40, n_iter=8)
    exps = [(1.0, 2.0), (1.5, 2.5), (2.0, 1.0), (0.5, 0.5), (1.0, 2.0), (3.0, 1.75), (0.0, 2.0), (1.25, 0.0)]
    qs = [dataclasses.replace(q, n_ants=6 + 5 * i, alpha=exps[i][0], beta=exps[i][1]) for i, q in enumerate(wl.queries)]
    ctx.load_workload(wl)
    ctx.set_params(**SCHEDULES[sched])
    res = ctx.solve_batch(qs)
    onet = orc.Net.from_workload(wl)
    for i, q in enumerate(qs):
        _compare(orc, onet, orc.Params(), q, res[i], ctx, i)

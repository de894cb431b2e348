"""Parity of the paper-literal pheromone variant (repulsive scores, unit deposits, unused-only
evaporation; Sec. 4.1, Fig. 3, Algorithm 2) and of saturated scores, GPU against the oracle bit for bit,
through the C ABI, for every kernel shape and both pheromone layouts."""
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
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


def _flag_sets(gm):
    return {"repulsive": gm.FLAG_REPULSIVE, "unit": gm.FLAG_UNIT_DEPOSIT, "unused": gm.FLAG_EVAP_UNUSED,
            "literal": gm.FLAG_PAPER_LITERAL}


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("which", ["repulsive", "unit", "unused", "literal"])
def test_grid10_literal_flags(gm, ctx, orc, which, sched):
    wl = W.grid10(n_ants=32, n_iter=15)
    ctx.load_workload(wl)
    flags = _flag_sets(gm)[which]
    ctx.set_params(**_with_flags(sched, flags | gm.FLAG_ANT_LOG))
    q = wl.queries[0]
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(flags=flags), q, r, ctx, 0, ctx.ant_log(0))


@pytest.mark.parametrize("lanes", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("lockstep", [True, False])
def test_grid10_literal_every_kernel_shape(gm, ctx, orc, lanes, lockstep):
    wl = W.grid10(n_ants=48, n_iter=12)
    ctx.load_workload(wl)
    flags = gm.FLAG_PAPER_LITERAL | (0 if lockstep else gm.FLAG_NO_LOCKSTEP)
    ctx.set_params(lanes_per_ant=lanes, flags=flags)
    q = Q(wl.queries[0].src, wl.queries[0].dst, 48, 12, 2.0, 1.0, 0.2, 17)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(flags=gm.FLAG_PAPER_LITERAL), q, r, ctx)


def test_grid64_literal_batch(gm, ctx, orc):
    """Four colonies of a literal-variant job in the default schedule, each equal to its solo oracle solve."""
    wl = W.grid64(n_queries=4, n_ants=128, n_iter=10)
    ctx.load_workload(wl)
    ctx.set_params(flags=gm.FLAG_PAPER_LITERAL)
    res = ctx.solve_batch(wl.queries)
    onet = orc.Net.from_workload(wl)
    for i, q in enumerate(wl.queries):
        _compare(orc, onet, orc.Params(flags=gm.FLAG_PAPER_LITERAL), q, res[i], ctx, i)


@pytest.mark.parametrize("sched", ["chains_default", "persistent", "sparse_tau"])
def test_saturated_attractive_scores(gm, ctx, orc, sched):
    """Two parallel routes, alpha = 8, no evaporation, unit deposits on the used roads only: the
    favoured road passes 2^48 (2^16 as a factor), where tau^8 saturates at FLT_MAX."""
    roads = [(0, 1, 512, 45), (0, 2, 520, 45), (1, 3, 512, 45), (2, 3, 512, 45)]
    net, sig, veh = NB.build(4, roads, bidirectional=False)
    onet = orc.Net(net, sig, veh)
    flags = gm.FLAG_UNIT_DEPOSIT | gm.FLAG_EVAP_UNUSED
    q = Q(0, 3, 1024, 72, 8.0, 1.0, 0.0, 21)
    o = orc.solve(onet, orc.Params(flags=flags), q)
    # even before the last iteration's deposits the favoured road held more than 2^48
    assert int(o["tau"].max()) - q.n_ants * 2**32 > 2**48
    ctx.load_graph(net)
    ctx.set_signals(sig)
    ctx.set_densities(veh)
    ctx.set_params(**_with_flags(sched, flags))
    r = ctx.solve_batch([q])[0]
    _compare(orc, onet, orc.Params(flags=flags), q, r, ctx)


@pytest.mark.parametrize("sched", ["chains_default", "sparse_tau", "persistent"])
def test_saturated_repulsive_scores(gm, ctx, orc, sched):
    """Repulsive alpha = 8 with strong evaporation: roads no ant uses fall below 2^16 (a factor above 2^16),
    so their scores saturate; the roulette then separates them by the heuristic alone."""
    wl = W.grid10(n_ants=32, n_iter=40)
    flags = gm.FLAG_REPULSIVE | gm.FLAG_UNIT_DEPOSIT
    q = Q(wl.queries[0].src, wl.queries[0].dst, 32, 40, 8.0, 1.0, 0.6, 23)
    onet = orc.Net.from_workload(wl)
    o = orc.solve(onet, orc.Params(flags=flags), q)
    assert int(o["tau"].min()) < 2**16
    ctx.load_workload(wl)
    ctx.set_params(**_with_flags(sched, flags))
    r = ctx.solve_batch([q])[0]
    _compare(orc, onet, orc.Params(flags=flags), q, r, ctx)


@pytest.mark.parametrize("exact", [False, True])
def test_random_initial_pheromone_repulsive(gm, ctx, orc, exact):
    """Philox-random initial pheromone read through the reciprocal word (and with the exact heuristic)."""
    wl = W.grid10(n_ants=32, n_iter=10)
    ctx.load_workload(wl)
    flags = gm.FLAG_RANDOM_TAU | gm.FLAG_REPULSIVE | (gm.FLAG_EXACT_H if exact else 0)
    ctx.set_params(flags=flags | gm.FLAG_ANT_LOG)
    q = Q(wl.queries[0].src, wl.queries[0].dst, 32, 10, 2.0, 1.0, 0.15, 77)
    r = ctx.solve_batch([q])[0]
    _compare(orc, orc.Net.from_workload(wl), orc.Params(flags=flags), q, r, ctx, 0, ctx.ant_log(0))

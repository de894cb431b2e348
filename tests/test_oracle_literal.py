"""Pins of the oracle's paper-literal variant (Sec. 4.1 bullets, Fig. 3, Algorithm 2) and of score
saturation: hand-worked picks with the first Philox draws, chi-square frequencies of the repulsive rule,
closed-form pheromone recurrences on a graph with a single route, and a one-iteration identity on grid10.
No GPU needed."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests import netbuild as NB
from tests.test_oracle_primitives import _exact_weights
from tests.test_oracle_solve import _expected_pick, _star

Q = W.Query
FMAX = np.float32(np.finfo(np.float32).max)


def test_score_saturates_at_largest_finite(orc):
    """tau = 2^63 is 2^31 as a factor: alpha = 4 gives 2^124 exactly, alpha >= 5 would overflow and
    saturates at FLT_MAX; the heuristic factor (<= 1) then scales the saturated value."""
    assert orc.score(2**63, 4, 1, 0) == np.float32(2.0**124)
    for a in (5, 6, 8):
        assert orc.score(2**63, a, 1, 0) == FMAX
    c = 3000
    eta = np.float32(1) / np.float32(c)
    assert orc.score(2**63, 8, c, 2) == FMAX * (eta * eta)
    # repulsive: tau = 1 (the smallest pheromone) is 2^32 as a factor, 2^256 at alpha = 8
    assert orc.score(1, 8, 1, 0, orc.FLAG_REPULSIVE) == FMAX
    assert orc.score(1, 3, 1, 0, orc.FLAG_REPULSIVE) == np.float32(2.0**96)
    # the saturated maximum still gives weights below 2^23
    w = orc.quantize(np.array([FMAX, np.float32(1.0), FMAX * np.float32(0.5)], np.float32))
    assert [int(v) for v in w] == _exact_weights([FMAX, np.float32(1.0), FMAX * np.float32(0.5)])
    assert int(w[0]) == 2**23 - 1 and int(w[1]) == 1 and int(w[2]) == 2**22 - 1


def test_repulsive_factor_is_rounded_reciprocal(orc):
    """The factor is 1/(tau/2^32) rounded once: exact for powers of two, nearest binary32 otherwise."""
    for tau, want in [(2**32, 1.0), (2**33, 0.5), (2**30, 4.0), (1, 2.0**32), (2**63, 2.0**-31)]:
        assert orc.tau_factor(tau, orc.FLAG_REPULSIVE) == np.float32(want)
    for tau in (3 * 2**32, 7 * 2**29, 2**32 + 12345, 987654321):
        tf = Fraction(float(np.float32(tau) * np.float32(2.0**-32)))
        got = Fraction(float(orc.tau_factor(tau, orc.FLAG_REPULSIVE)))
        exact = 1 / tf
        # nearest: no binary32 neighbour of got is closer to 1/tf
        lo = Fraction(float(np.nextafter(np.float32(got), np.float32(0))))
        hi = Fraction(float(np.nextafter(np.float32(got), np.float32(np.inf))))
        assert abs(got - exact) <= abs(lo - exact) and abs(got - exact) <= abs(hi - exact)


def _star_tau(net, taus_out_of_0):
    tau = np.full(net.n_edges, 2**32, np.uint64)
    for head, t in zip((1, 2, 3), taus_out_of_0):
        tau[NB.edge_id(net, 0, head)] = t
    return tau


def test_repulsive_hand_worked_picks(orc):
    """Pheromone 1, 2, 4 on roads 0->1, 0->2, 0->3, alpha = 1, beta = 0: the factors are 1, 1/2, 1/4,
    so the weights are 2^22, 2^21, 2^20 (attractive: 2^20, 2^21, 2^22). Each ant's first road follows
    the roulette over those weights with its own Philox draw."""
    net, sig, veh = _star()
    onet = orc.Net(net, sig, veh)
    tau = _star_tau(net, [2**32, 2**33, 2**34])
    for flags, weights in [(orc.FLAG_REPULSIVE, [2**22, 2**21, 2**20]), (0, [2**20, 2**21, 2**22])]:
        picks = []
        for ant in range(200):
            w = orc.walk_one(onet, orc.Params(flags=flags), Q(0, 4, 200, 1, 1.0, 0.0, 0.1, 41), tau, it=0, ant=ant)
            pick = _expected_pick(orc, weights, 41, 0, ant, 0)
            assert int(net.col[w["route_edges"][0]]) == 1 + pick
            picks.append(pick)
        assert set(picks) == {0, 1, 2}


def test_repulsive_frequencies_chi_square(orc):
    """P(road i) is proportional to tau_i^-alpha: 4/7, 2/7, 1/7 at alpha = 1; 16/21, 4/21, 1/21 at alpha = 2."""
    from scipy.stats import chisquare

    net, sig, veh = _star()
    onet = orc.Net(net, sig, veh)
    tau = _star_tau(net, [2**32, 2**33, 2**34])
    for a, probs in [(1.0, [4 / 7, 2 / 7, 1 / 7]), (2.0, [16 / 21, 4 / 21, 1 / 21])]:
        counts = [0, 0, 0]
        n = 6000
        for ant in range(n):
            w = orc.walk_one(onet, orc.Params(flags=orc.FLAG_REPULSIVE), Q(0, 4, n, 1, a, 0.0, 0.1, 6), tau, it=0,
                             ant=ant)
            counts[int(net.col[w["route_edges"][0]]) - 1] += 1
        assert chisquare(counts, [n * p for p in probs]).pvalue > 1e-4, counts


def _line_with_spur():
    """0 - 1 - 2 - 3 with a spur 1 - 4 (both directions). Node 4 is a dead end for an ant coming from
    1, so the only route 0 -> 3 is 0, 1, 2, 3; an ant that enters the spur steps back to 1, which
    takes it 5 moves in all instead of 3."""
    roads = [(0, 1, 512, 45), (1, 2, 512, 45), (2, 3, 512, 45), (1, 4, 512, 45)]
    coords = [(0, 0), (512, 0), (1024, 0), (1536, 0), (512, 512)]
    return NB.build(5, roads, coords)


@pytest.mark.parametrize("flags", [0, 64, 128, 64 | 128, 32 | 64 | 128])
def test_single_route_closed_form(orc, flags):
    """Every successful ant takes the same three roads with the same T. Per iteration with n successes:
    route roads: tau <- evap(tau) + n*delta, or with unused-only evaporation tau + n*delta when n > 0
    and evap(tau) when n = 0; every other road evaporates every iteration. delta = 1.0 with unit
    deposits, else floor(max(h(src),1) * 2^32 / T). A cap of 4 moves makes the ants that enter the
    spur fail, so iterations with no success occur; beta = 0 keeps the spur as likely as the road on
    (the heuristic would rule it out)."""
    net, sig, veh = _line_with_spur()
    onet = orc.Net(net, sig, veh)
    q = Q(0, 3, 6, 12, 1.0, 0.0, 0.25, 9)
    prm = orc.Params(flags=flags, max_steps=4)
    r = orc.solve(onet, prm, q, want_log=True)
    st, _, moves, _, _ = orc.log_fields(r["log"])
    log = r["log"]
    ok = st == 0
    assert ok.any() and (~ok).any()  # ants that enter the spur run out of moves
    assert (moves[ok] == 3).all() and (st[~ok] == orc.ANT_STEP_CAP).all()
    T = {int(t) for t in log[:, :, 2][ok]}
    assert len(T) == 1
    T = T.pop()
    h_src = int(orc.prepare(onet, prm, 3)["h"][0])
    delta = 2**32 if flags & 64 else (max(h_src, 1) << 32) // T
    rf = orc.rho_fix(q.rho)
    route = {NB.edge_id(net, 0, 1), NB.edge_id(net, 1, 2), NB.edge_id(net, 2, 3)}
    t_route, t_other = 2**32, 2**32
    for it in range(q.n_iter):
        n = int(ok[it].sum())
        if flags & 128:
            t_route = t_route + n * delta if n else orc.evaporate(t_route, rf)
        else:
            t_route = orc.evaporate(t_route, rf) + n * delta
        t_other = orc.evaporate(t_other, rf)
    for e in range(net.n_edges):
        assert int(r["tau"][e]) == (t_route if e in route else t_other), e


def test_literal_one_iteration_identity_grid10(orc):
    """One iteration of the paper-literal variant from tau = 1.0: a road some successful ant used holds
    1 + (its number of uses), every other road evap(1.0); so the number of used roads is the number of
    roads above 1.0, and the sum over roads is fixed by the ants' step counts."""
    wl = W.grid10(n_ants=32, n_iter=1)
    onet = orc.Net.from_workload(wl)
    q = wl.queries[0]
    r = orc.solve(onet, orc.Params(flags=orc.FLAG_PAPER_LITERAL), q, want_log=True)
    st, length, _, _, _ = orc.log_fields(r["log"][0])
    uses = int(length[st == 0].sum())
    assert uses > 0
    tau = r["tau"].astype(object)
    low = orc.evaporate(2**32, orc.rho_fix(q.rho))
    used = [t for t in tau if t > 2**32]
    assert all(t == low for t in tau if t <= 2**32)
    assert all(t % 2**32 == 0 for t in used)
    assert sum(used) == len(used) * 2**32 + uses * 2**32
    assert len(used) + sum(1 for t in tau if t == low) == wl.net.n_edges


def test_repulsive_unit_deposits_balance_parallel_routes(orc):
    """Three equal parallel routes, alpha = 1, beta = 0, no evaporation: each deposit makes a road less
    likely to be chosen again, so the use counts stay close to each other; the attractive rule with the
    same deposits lets one route run away more than the repulsive one ever does."""
    roads = [(0, 1, 512, 45), (0, 2, 512, 45), (0, 3, 512, 45), (1, 4, 512, 45), (2, 4, 512, 45), (3, 4, 512, 45)]
    net, sig, veh = NB.build(5, roads, bidirectional=False)
    onet = orc.Net(net, sig, veh)
    q = Q(0, 4, 16, 40, 1.0, 0.0, 0.0, 12)
    spread = {}
    for flags in (orc.FLAG_PAPER_LITERAL, orc.FLAG_UNIT_DEPOSIT | orc.FLAG_EVAP_UNUSED):
        r = orc.solve(onet, orc.Params(flags=flags), q)
        uses = [int(r["tau"][NB.edge_id(net, 0, h)]) // 2**32 - 1 for h in (1, 2, 3)]
        assert sum(uses) == q.n_ants * q.n_iter
        spread[flags] = max(uses) - min(uses)
    assert spread[orc.FLAG_PAPER_LITERAL] <= 0.05 * q.n_ants * q.n_iter
    assert spread[orc.FLAG_UNIT_DEPOSIT | orc.FLAG_EVAP_UNUSED] > spread[orc.FLAG_PAPER_LITERAL]

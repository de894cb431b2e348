"""Pins of the CPU oracle's building blocks against values fixed outside the oracle.

Each test checks one oracle function against something it does not itself compute: published
known-answer vectors, Python's exact integer/rational arithmetic, hand-worked numbers, or a brute-force
simulation. Nothing here needs a GPU.
"""
import math
import os
import random
from fractions import Fraction

import numpy as np

from tests import netbuild as NB

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------ Philox
def test_philox_known_answers(orc):
    """Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            assert orc.philox(w[0:4], w[4:6]) == tuple(w[6:10])
            rows += 1
    assert rows == 3


def test_philox_counter_sensitivity(orc):
    """Every counter and key word changes the output (no word is ignored or aliased)."""
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert orc.philox(c, [5, 6]) != base
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert orc.philox([1, 2, 3, 4], k) != base


# ------------------------------------------------------------------------------------------ isqrt
def test_isqrt_matches_python(orc):
    rng = random.Random(7)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, 2**32 - 1, 2**32, 2**62, 2**63 - 1, 2**64 - 1]
    for r in range(1, 200):
        vals += [r * r - 1, r * r, r * r + 1]
    big = [(2**32 - 1) ** 2, (2**32 - 1) ** 2 - 1, (3037000499) ** 2, (3037000499) ** 2 - 1]
    vals += big + [rng.getrandbits(64) for _ in range(20000)] + [rng.getrandbits(40) for _ in range(5000)]
    for v in vals:
        assert orc.isqrt(v) == math.isqrt(v), v


# ------------------------------------------------------------------------------------------ roads
def test_free_flow_hand_worked(orc):
    # 100 m at 50 km/h = 100 / (50/3.6) s = 7.2 s
    assert orc.free_flow_ms(1000, 50) == 7200
    # 100 m at 70 km/h = 5.142857 s -> 5143 ms (rounded)
    assert orc.free_flow_ms(1000, 70) == 5143
    # 1 m at 1 km/h = 3.6 s
    assert orc.free_flow_ms(10, 1) == 3600
    # 0.1 m at 70 km/h = 5.14 ms -> 5 ms ; 1 dm at 1000 km/h = 0.36 ms -> at least 1 ms
    assert orc.free_flow_ms(1, 70) == 5
    assert orc.free_flow_ms(1, 1000) == 1
    # 51.2 m at 45 km/h = 4.096 s (chosen to be exact in binary)
    assert orc.free_flow_ms(512, 45) == 4096
    # clamp at 2^26 ms
    assert orc.free_flow_ms(2**32 - 1, 1) == 2**26


def test_capacity_hand_worked(orc):
    assert orc.capacity(3, 1000) == 40  # 3 lanes x 100 m / 7.5 m
    assert orc.capacity(1, 75) == 1
    assert orc.capacity(1, 50) == 1  # shorter than one car: still holds one
    assert orc.capacity(2, 150) == 4


def test_edge_time_hand_worked_and_monotone(orc):
    assert orc.edge_time_ms(7200, 40, 0) == 7200  # empty road: free flow
    assert orc.edge_time_ms(7200, 40, 20) == 14400  # half full: twice free flow
    assert orc.edge_time_ms(7200, 40, 30) == 28800  # 3/4 full: 4x
    # nearly jammed / over capacity: denominator floors at cap/20 = 2 -> 20x free flow
    assert orc.edge_time_ms(7200, 40, 39) == 144000
    assert orc.edge_time_ms(7200, 40, 1000) == 144000
    # tiny capacity: floor 1 -> cap x free flow
    assert orc.edge_time_ms(100, 3, 5) == 300
    for cap in (1, 2, 5, 19, 20, 21, 40, 400):
        prev = 0
        for n in range(0, 2 * cap + 3):
            t = orc.edge_time_ms(1000, cap, n)
            assert t >= prev and t >= 1000
            prev = t


def test_queue_delay_hand_worked(orc):
    assert orc.queue_delay_ms(10, 2000, 3, True) == 6666  # 10 vehicles, 2 s headway, 3 lanes
    assert orc.queue_delay_ms(10, 2000, 3, False) == 0
    assert orc.queue_delay_ms(0, 2000, 1, True) == 0


# ------------------------------------------------------------------------------------------ signals
def _green_phase_at(tms, cycle, offset, green, order):
    """Which phase shows green at absolute time tms (simulated from the programme)."""
    c = (tms - offset) % cycle
    acc = 0
    for p in order:
        if acc <= c < acc + green[p]:
            return p
        acc += green[p]
    raise AssertionError("greens must cover the cycle")


def test_signal_wait_matches_simulation(orc):
    rng = random.Random(3)
    for _ in range(400):
        P = rng.randint(1, 4)
        green = [rng.randint(1, 9) for _ in range(P)]
        cycle = sum(green)
        offset = rng.randrange(cycle)
        order = list(range(P))
        rng.shuffle(order)
        phase = rng.randrange(P)
        arr = rng.randrange(0, 10 * cycle + 5)
        k = 0
        while _green_phase_at(arr + k, cycle, offset, green, order) != phase:
            k += 1
        assert orc.signal_wait_ms(arr, cycle, offset, green, order, P, phase) == k


def test_signal_wait_large_times(orc):
    # 90 s cycle, phase 0 green 40 s from offset 10 s in default order; arrival 2^31 ms
    arr = 2**31
    c = (arr - 10_000) % 90_000
    expect = 0 if c < 40_000 else 90_000 - c
    assert orc.signal_wait_ms(arr, 90_000, 10_000, [40_000, 50_000], [0, 1], 2, 0) == expect


def _order_by_sort_key(P, Q, Th, red, Tmax):
    """The preemption rule restated as one sort: selected phases first (by the rule that fired),
    then non-empty queues in default order, then empty queues in default order."""
    over = [p for p in range(P) if Q[p] > Th[p]]
    starved = [p for p in range(P) if red[p] > Tmax]
    if over:
        sel = {p: (-Q[p], p) for p in over}
    elif starved:
        sel = {p: (-red[p], p) for p in starved}
    else:
        nz = [p for p in range(P) if Q[p] > 0]
        sel = {}
        if nz:
            m = max(Q[p] for p in nz)
            sel = {min(p for p in nz if Q[p] == m): (0, 0)}
    key = lambda p: (0,) + sel[p] if p in sel else ((1, 0, p) if Q[p] > 0 else (2, 0, p))
    return sorted(range(P), key=key)


def test_phase_order_exhaustive_small(orc):
    """All queue patterns in {0..3}^P for P <= 4, thresholds 1 or 2, with/without a starved phase."""
    import itertools

    for P in range(1, 5):
        for Q in itertools.product(range(4), repeat=P):
            for th in (1, 2):
                Th = [th] * P
                for red in ([0] * P, [0] * (P - 1) + [100], [100] * P):
                    got = orc.phase_order(P, list(Q), Th, red, 50)
                    assert got == _order_by_sort_key(P, list(Q), Th, red, 50), (P, Q, th, red)
                    assert sorted(got) == list(range(P))


def test_phase_order_random_up_to_8(orc):
    rng = random.Random(11)
    for _ in range(3000):
        P = rng.randint(1, 8)
        Q = [rng.choice([0, 0, 1, 2, 5, 9]) for _ in range(P)]
        Th = [rng.randint(0, 8) for _ in range(P)]
        red = [rng.choice([0, 10, 60, 61, 200]) for _ in range(P)]
        assert orc.phase_order(P, Q, Th, red, 60) == _order_by_sort_key(P, Q, Th, red, 60)


def test_phase_order_paper_cases(orc):
    """Narrative cases of the preemptive rule (Sec. 4.1-4.2)."""
    # no queue anywhere: the default order is kept
    assert orc.phase_order(4, [0, 0, 0, 0], [5] * 4, [0] * 4, 60) == [0, 1, 2, 3]
    # the phase with the longest queue is served first, empty phases are skipped to the end
    assert orc.phase_order(4, [2, 0, 4, 1], [5] * 4, [0] * 4, 60) == [2, 0, 3, 1]
    # a queue above its threshold takes precedence over a longer-waiting phase
    assert orc.phase_order(3, [1, 7, 3], [5, 5, 5], [99, 0, 0], 60) == [1, 0, 2]
    # no queue above threshold: the starved phase goes first
    assert orc.phase_order(3, [1, 4, 3], [5, 5, 5], [0, 0, 99], 60) == [2, 0, 1]


def test_queue_threshold_is_three_quarters_of_storage(orc):
    """Comp_Thres on a hand-built junction: the phase-0 approach stores 3 * 2500 dm / 7.5 m = 100
    vehicles, so its threshold is 75; the phase-1 approach stores 1000 and holds 80. Up to 75 vehicles
    on phase 0 no queue is over, and the longer queue (phase 1) goes first. From 76 on, phase 0 is over
    its threshold and takes precedence."""
    roads = [(0, 2, 2500, 50, 3, 0), (1, 2, 25000, 50, 3, 1)]
    for n0, want in [(70, [1, 0]), (75, [1, 0]), (76, [0, 1])]:
        net, sig, veh = NB.build(3, roads, signals={2: (60000, 0, [30000, 30000])},
                                 vehicles={(0, 2): n0, (1, 2): 80}, bidirectional=False)
        order = orc.queue_preempt(orc.Net(net, sig, veh))
        assert list(order[2][:2]) == want, n0
        assert list(order[2][2:]) == [2, 3, 4, 5, 6, 7]


# ------------------------------------------------------------------------------------------ heuristic
def test_heuristic_hand_worked(orc):
    # 300 m x 400 m offset = 500 m straight line; at 100 km/h that is 18 s. kappa = floor(360*2^16/100)
    k = orc.kappa(100)
    assert k == 235929
    assert orc.heuristic_ms(3000, 4000, 0, 0, k) == (5000 * 235929) >> 16 == 17999
    assert orc.heuristic_ms(7, 7, 7, 7, k) == 0
    # never above the exact straight-line time (admissible)
    rng = random.Random(5)
    for _ in range(2000):
        x, y, xd, yd = (rng.randint(-10**6, 10**6) for _ in range(4))
        v = rng.choice([30, 45, 70, 105])
        h = orc.heuristic_ms(x, y, xd, yd, orc.kappa(v))
        exact = Fraction(math.isqrt((x - xd) ** 2 + (y - yd) ** 2) * 360, v)
        assert h <= exact and exact - h < Fraction(math.isqrt((x - xd) ** 2 + (y - yd) ** 2) + 65536, 65536)


# ------------------------------------------------------------------------------------------ scores
def _exact_weights(scores):
    """w_i = max(1, floor(s_i * 2^(22 - E))), E = floor(log2(max s)); exact rational arithmetic."""
    fr = [Fraction(float(s)) for s in scores]
    m = max(fr)
    if m == 0:
        return [1] * len(fr)
    E = m.numerator.bit_length() - m.denominator.bit_length()
    if Fraction(2) ** E > m:
        E -= 1
    assert Fraction(2) ** E <= m < Fraction(2) ** (E + 1)
    return [max(1, math.floor(f * Fraction(2) ** (22 - E))) for f in fr]


def test_quantize_matches_exact_rationals(orc):
    rng = np.random.default_rng(1)
    cases = [np.array([0.0, 0.0], np.float32), np.array([1.0], np.float32),
             np.array([2.0**-11, 2.0**-12, 2.0**-13], np.float32),
             np.array([1e-45, 3e-45, 0.0], np.float32),  # subnormal maximum
             np.array([3.4e38, 1e-30, 1.0], np.float32)]
    for _ in range(3000):
        n = int(rng.integers(1, 9))
        e = rng.integers(-149, 60, size=n).astype(np.float64)
        s = (rng.random(n) * np.exp2(e)).astype(np.float32)
        if rng.random() < 0.2:
            s[rng.integers(0, n)] = 0
        cases.append(s)
    for s in cases:
        w = orc.quantize(s)
        assert [int(v) for v in w] == _exact_weights(s), s
        assert int(w.max()) < 2**23 and int(w.min()) >= 1


def test_score_binary32_order(orc):
    """s = (tau/2^32)^alpha * (1/c)^beta, one binary32 rounding per operation (numpy float32 ops)."""
    f32 = np.float32
    rng = random.Random(2)
    for _ in range(3000):
        tau = rng.choice([1, 2**32, 3 * 2**31, rng.randrange(1, 2**24) << rng.randrange(0, 40)])
        c = rng.randrange(1, 2**24)
        a, b = rng.randint(0, 4), rng.randint(0, 4)
        tf = f32(tau) * f32(2.0**-32)  # tau < 2^64 with <= 24 significant bits: exact conversion
        eta = f32(1.0) / f32(c)
        pa = f32(1.0)
        if a:
            pa = tf
            for _ in range(a - 1):
                pa = f32(pa * tf)
        pb = f32(1.0)
        if b:
            pb = eta
            for _ in range(b - 1):
                pb = f32(pb * eta)
        expect = f32(pa * pb)
        got = orc.score(tau, a, c, b)
        assert got.tobytes() == expect.tobytes(), (tau, a, c, b)


def test_roulette_hand_worked(orc):
    w = [2**29, 2**28, 2**30]  # prefix sums 2^29, 3*2^28, 7*2^28 ; S = 7*2^28
    S = 7 * 2**28
    # r = floor(rnd*S/2^64): choose rnd so that r hits both sides of each boundary
    for r, expect in [(0, 0), (2**29 - 1, 0), (2**29, 1), (3 * 2**28 - 1, 1), (3 * 2**28, 2), (S - 1, 2)]:
        rnd = -(-(r << 64) // S)  # smallest rnd with floor(rnd*S/2^64) == r
        assert (rnd * S) >> 64 == r
        assert orc.roulette_pick(w, rnd) == expect
    assert orc.roulette_pick(w, 2**64 - 1) == 2


def test_roulette_chi_square(orc):
    """Chosen-index frequencies over Philox draws follow w_i / S."""
    from scipy.stats import chisquare

    w = [5, 1, 3, 7, 1]
    counts = [0] * len(w)
    for i in range(40000):
        o = orc.philox([i, 7, 0, 0], [123, 0])
        counts[orc.roulette_pick(w, o[0] | (o[1] << 32))] += 1
    S = sum(w)
    exp = [40000 * x / S for x in w]
    assert chisquare(counts, exp).pvalue > 1e-4


# ------------------------------------------------------------------------------------------ pheromone
def test_rho_fix_and_evaporation_hand_worked(orc):
    # 0.1f = 13421773 * 2^-27 exactly, so 0.1f * 2^32 = 13421773 * 32 = 429496736 (an integer)
    assert orc.rho_fix(0.1) == 429496736
    assert orc.rho_fix(0.0) == 0
    assert orc.rho_fix(0.5) == 2**31
    r = 429496736
    # 1.0 (=2^32) loses exactly rho_fix
    assert orc.evaporate(2**32, r) == 2**32 - 429496736 == 3865470560
    # 10.0 loses 10*rho_fix = 4294967360
    assert orc.evaporate(10 * 2**32, r) == 42949672960 - 4294967360
    # the smallest pheromone never evaporates below 1
    assert orc.evaporate(1, r) == 1
    assert orc.evaporate(7, 2**32 - 1) >= 1


def test_random_tau_init_range(orc):
    t = orc.init_tau(5000, 99, flags=1)
    assert t.min() >= 2**31 and t.max() < 2**31 + 2**32
    assert len(set(t.tolist())) > 4990
    assert (orc.init_tau(10, 99, flags=0) == 2**32).all()
    # word 0 of Philox(counter = (road, 0, 0, 1), key = seed)
    assert int(t[17]) == 2**31 + orc.philox([17, 0, 0, 1], [99, 0])[0]

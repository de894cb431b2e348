"""Pins of the oracle's score for non-integer alpha / beta: its binary32 log2 and exp2 against the
mathematics (exact series constants, exact powers of two, error bounds against double precision), the
resulting score against double-precision powers, and the roulette frequencies it gives. No GPU needed.

Error bounds (derived from the operation counts, with a margin, and checked here): log2 within
2^-22 |log2 x|; exp2 within 2^-22 relative for normal results; the score within
2^-21 (alpha |log2 f| + beta log2 c + 1) relative, f the pheromone factor, c the cost in ms."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from paper_2010_14244_gb300 import workloads as W
from tests.test_oracle_literal import _star_tau
from tests.test_oracle_solve import _star

Q = W.Query
FMAX = np.float32(np.finfo(np.float32).max)


def _round_f32(x: Fraction) -> float:
    """The binary32 nearest to a positive rational (ties to even), by exact arithmetic."""
    e = x.numerator.bit_length() - x.denominator.bit_length()
    while Fraction(2) ** e > x:
        e -= 1
    while Fraction(2) ** (e + 1) <= x:
        e += 1
    q = x / Fraction(2) ** (e - 23)
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2):
        n += 1
    return float(Fraction(n) * Fraction(2) ** (e - 23))


def test_series_constants_are_nearest_binary32(orc):
    getcontext().prec = 60
    ln2 = Fraction(Decimal(2).ln())
    want = [Fraction(1, 3), Fraction(1, 5), Fraction(1, 7), Fraction(1, 9), 2 / ln2]
    want += [Fraction(1)] + [ln2 ** k / math.factorial(k) for k in range(1, 9)]
    got = orc.frac_constants()
    assert [float(g) for g in got] == [_round_f32(w) for w in want]


def test_log2_exact_powers_and_bound(orc):
    for k in range(-126, 128):
        assert orc.log2f(2.0 ** k) == np.float32(k)
    rng = np.random.default_rng(3)
    xs = (rng.random(60000) * np.exp2(rng.integers(-60, 60, 60000))).astype(np.float32)
    xs = np.concatenate([xs, np.float32(1) + (rng.random(5000) * 1e-3).astype(np.float32),
                         np.float32(1) - (rng.random(5000) * 1e-3).astype(np.float32),
                         np.float32([np.sqrt(2), np.nextafter(np.float32(np.sqrt(2)), 2), 1 / np.sqrt(2)])])
    for x in xs[xs >= 2.0 ** -126]:
        t = math.log2(float(x))
        assert abs(float(orc.log2f(x)) - t) <= 2.0 ** -22 * abs(t), x


def test_exp2_exact_powers_saturation_and_bound(orc):
    for k in range(-149, 128):
        assert float(orc.exp2f(k)) == 2.0 ** k
    for L in (128.0, 128.5, 1000.0):
        assert orc.exp2f(L) == FMAX
    top = float(orc.exp2f(np.nextafter(np.float32(128), np.float32(0))))
    assert math.isfinite(top) and 2.0 ** 127 * 1.9999 < top <= float(FMAX)
    assert orc.exp2f(-150.5) == 0 and orc.exp2f(-1e9) == 0
    rng = np.random.default_rng(4)
    for L in rng.uniform(-126, 128, 60000).astype(np.float32):
        t = 2.0 ** float(L)
        if t < float(FMAX):
            assert abs(float(orc.exp2f(L)) - t) <= 2.0 ** -22 * t, L


def test_score_against_double_powers(orc):
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(40000):
        tau = max(1, int(rng.integers(1, 2 ** 63)) >> int(rng.integers(0, 62)))
        c = max(1, int(rng.integers(1, 2 ** 29)) >> int(rng.integers(0, 28)))
        a, b = float(np.float32(rng.uniform(0, 8))), float(np.float32(rng.uniform(0, 8)))
        flags = orc.FLAG_REPULSIVE if rng.random() < 0.3 else 0
        f = float(orc.tau_factor(tau, flags))
        cf = float(np.float32(c))
        L = a * math.log2(f) - b * math.log2(cf)
        got = float(orc.score_frac(tau, a, c, b, flags))
        if L >= 128.01:
            assert got == float(FMAX)
        elif -125 < L < 127.99:
            t = 2.0 ** L
            assert abs(got - t) <= 2.0 ** -21 * (a * abs(math.log2(f)) + b * math.log2(cf) + 1) * t
            checked += 1
    assert checked > 25000


def test_integer_exponents_agree_with_repeated_multiplication(orc):
    """Both forms compute f^a (1/c)^b; for integer exponents they agree within the bound."""
    rng = np.random.default_rng(6)
    for _ in range(3000):
        tau = max(1, int(rng.integers(1, 2 ** 40)))
        c = int(rng.integers(1, 2 ** 24))
        a, b = int(rng.integers(0, 5)), int(rng.integers(0, 5))
        s_int = float(orc.score(tau, a, c, b))
        s_frac = float(orc.score_frac(tau, a, c, b))
        f = float(orc.tau_factor(tau))
        if s_int > 2.0 ** -120:
            assert abs(s_frac - s_int) <= 2.0 ** -20 * (a * abs(math.log2(f)) + b * math.log2(c) + 1 + a + b) * s_int


@pytest.mark.parametrize("alpha,beta,flags", [(0.5, 0.0, 0), (1.5, 0.0, 32), (0.0, 1.5, 0), (0.5, 2.5, 0)])
def test_fractional_exponent_frequencies_chi_square(orc, alpha, beta, flags):
    """Star graph: pheromone 1, 2, 4 and costs 4096, 8192, 2048 ms (no signals, h = 0) on the three
    first roads. P(road i) is proportional to f_i^alpha * c_i^-beta."""
    from scipy.stats import chisquare

    net, sig, veh = _star()
    onet = orc.Net(net, sig, veh)
    tau = _star_tau(net, [2 ** 32, 2 ** 33, 2 ** 34])
    f = np.array([1.0, 2.0, 4.0])
    if flags:
        f = 1 / f
    c = np.array([4096.0, 8192.0, 2048.0])
    p = f ** alpha * c ** -beta
    p /= p.sum()
    n = 6000
    counts = [0, 0, 0]
    for ant in range(n):
        w = orc.walk_one(onet, orc.Params(flags=flags), Q(0, 4, n, 1, alpha, beta, 0.1, 8), tau, it=0, ant=ant)
        counts[int(net.col[w["route_edges"][0]]) - 1] += 1
    assert chisquare(counts, n * p).pvalue > 1e-4, (counts, n * p)


def test_fractional_colony_runs(orc):
    """A full colony with non-integer exponents finds routes on grid10 and keeps the pheromone identities."""
    wl = W.grid10(n_ants=32, n_iter=10)
    q = Q(wl.queries[0].src, wl.queries[0].dst, 32, 10, 1.25, 2.5, 0.1, 4)
    r = orc.solve(orc.Net.from_workload(wl), orc.Params(), q)
    assert r["status"] == 0 and r["n_success"] > 0
    assert int(r["tau"].min()) >= 1

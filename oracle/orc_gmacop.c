/*
 * GMACO-P CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the MACO-P route colony (Jindal & Bedi, "GMACO-P: GPU
 * assisted Preemptive MACO algorithm for enabling Smart Transportation", Sec. 4, Fig. 3, Algorithms 1-2)
 * under the readings fixed for the paper's unstated constants (integer milliseconds and decimetres,
 * Q32.32 pheromone, Philox4x32-10 draws, FP32 scores without FMA). It exists to check the CUDA library
 * result-for-result. Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it; the CUDA library never calls it and shares no source with it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC (see oracle/build.py).
 * Every float operation below is a single IEEE-754 binary32 operation rounded to nearest even.
 *
 * Parity status of each function (what pins it is listed in the tests):
 *   orc_philox4x32_10     pinned: Random123 known-answer vectors (Salmon et al., SC'11)
 *   orc_isqrt64           pinned: Python math.isqrt
 *   orc_free_flow_ms ...  pinned: hand-worked values and monotonicity (the paper gives no formula)
 *   orc_signal_wait_ms    pinned: millisecond-by-millisecond signal simulation
 *   orc_phase_order       pinned: an independent rule-by-rule enumeration over small tables
 *   orc_score_f           pinned: hand-worked scores, saturation at FLT_MAX, reciprocal pheromone
 *   orc_log2, orc_exp2    pinned: error bounds against double-precision log2 / exp2, exact special
 *                         values, series constants against their exact values (Python fractions)
 *   orc_score_frac        pinned: error bound against double-precision powers, chi-square frequencies
 *   orc_exact_heuristic   pinned: scipy's Dijkstra on the reversed graph, brute force over simple paths,
 *                         the clamp for nodes that cannot reach the destination
 *   orc_queue_preempt     pinned: a hand-built junction on both sides of the 3/4-storage threshold
 *   orc_heuristic_ms      pinned: hand-worked straight-line bounds
 *   orc_quantize          pinned: exact rational arithmetic (Python fractions)
 *   orc_roulette_pick     pinned: hand-worked picks, 128-bit products, chi-square frequencies
 *   orc_rho_fix, orc_evaporate  pinned: hand-worked values, tau never below 1
 *   orc_init_tau          pinned: word 0 of the Philox block keyed by the road, its range
 *   orc_walk_one          pinned: hand-worked single-ant steps and steps back at dead ends, chi-square
 *                         frequency checks
 *   orc_solve             pinned: Dijkstra / time-dependent Dijkstra / brute-force simple-path
 *                         enumeration on tiny graphs, route validity, pheromone conservation identity,
 *                         closed forms of the unit-deposit / unused-only-evaporation variant, the step
 *                         and time caps; the best route on large graphs is parity-unpinned (a
 *                         metaheuristic optimum)
 *   orc_tick              pinned: a hand-worked junction, a millisecond simulation of the programme,
 *                         conservation of vehicles, sinks, red-time growth and saturation
 * A test plants 67 single mistakes in copies of this file; each fails the pins of the part it changes.
 */
#include <float.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_PHASES 8
#define ORC_TIME_CLAMP (1u << 26) /* edge times, queue delays: at most 2^26 ms */
#define ORC_H_CLAMP (1u << 28)    /* heuristic lower bound: at most 2^28 ms */
#define ORC_T_CAP (1u << 30)      /* an ant whose elapsed time exceeds 2^30 ms fails */
#define ORC_DEFAULT_HSAT 2000u
#define ORC_THR_OFF 0xFFFFFFFFu
#define ORC_FLAG_RANDOM_TAU 1u
/* The paper's own MACO-P variant (Sec. 4.1 bullets, Fig. 3, Algorithm 2), one reading per flag: */
#define ORC_FLAG_REPULSIVE 32u    /* prefer less pheromone: the score reads 1/tau in place of tau */
#define ORC_FLAG_UNIT_DEPOSIT 64u /* Ph_road++: a successful ant adds exactly 1.0 to each road it used */
#define ORC_FLAG_EVAP_UNUSED 128u /* deposits first, then only roads without a deposit evaporate */
#define ORC_FLAG_EXACT_H 256u     /* Calc_Dist exactly: least congested travel time to the destination */

enum {
    ORC_OK = 0,
    ORC_ERR_INVALID = 1,
    ORC_ERR_NO_ROUTE = 2,
    ORC_ERR_OOM = 3,
    ORC_ERR_UNSUPPORTED = 6,
    ORC_ERR_BUFFER = 7,
};

enum { ANT_SUCCESS = 0, ANT_DEAD_END = 1, ANT_STEP_CAP = 2, ANT_TIME_CAP = 3 };

typedef struct {
    uint32_t n_nodes, n_edges;
    const uint32_t *row_ptr, *col, *length_dm;
    const uint16_t *speed_kmh;
    const uint8_t *lanes;
    const int32_t *x_dm, *y_dm;
    const uint8_t *n_phases;
    const uint32_t *cycle_ms, *offset_ms, *green_ms; /* green_ms: node*8 + phase */
    const uint8_t *edge_phase;
    const uint32_t *vehicles;
    const uint32_t *red_ms; /* node*8 + phase red-time accumulators, NULL = all zero */
} orc_net;

typedef struct {
    uint32_t max_steps;    /* moves per ant (forward and back); 0 = min(2(N-1), 4096) */
    uint32_t h_sat_ms;     /* 0 = 2000 ms saturation headway */
    uint32_t thr_permille; /* occupancy threshold in vehicles per 1000 capacity; 0xFFFFFFFF = off */
    uint32_t flags;        /* ORC_FLAG_* */
    uint32_t t_dep_ms;     /* departure clock, below 2^30 */
    uint32_t reserved;
} orc_params;

typedef struct {
    uint32_t src, dst, n_ants, n_iter;
    float alpha, beta, rho;
    uint32_t reserved;
    uint64_t seed;
} orc_query;

typedef struct {
    int32_t status;
    uint32_t route_len;
    uint64_t travel_ms, wait_ms, ant_steps, n_success;
    uint32_t best_iter, best_ant;
} orc_result;

/* ------------------------------------------------------------------------------------------------ */
/* Philox4x32-10, from its definition in Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications feeding a fixed word         */
/* permutation, with a Weyl-sequence key schedule between rounds.                                      */
/* ------------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* key increments (golden ratio, sqrt(3)-1) */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* 64-bit draw of the construction stream: key = seed, counter = (iteration, ant, step, 0). */
static uint64_t draw64(uint64_t seed, uint32_t it, uint32_t ant, uint32_t step, uint32_t stream)
{
    uint32_t c[4] = {it, ant, step, stream};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(c, k, o);
    return (uint64_t)o[0] | ((uint64_t)o[1] << 32);
}

/* floor(sqrt(n)) by the classic bit-pair (digit-by-digit) method. */
uint64_t orc_isqrt64(uint64_t n)
{
    uint64_t root = 0;
    uint64_t bit = (uint64_t)1 << 62;
    while (bit > n)
        bit >>= 2;
    while (bit != 0) {
        if (n >= root + bit) {
            n -= root + bit;
            root = (root >> 1) + bit;
        } else {
            root >>= 1;
        }
        bit >>= 2;
    }
    return root;
}

/* ------------------------------------------------------------------------------------------------ */
/* Road attributes (G(N,E) of Fig. 3; densities from road sensors, Sec. 4.2).                          */
/* ------------------------------------------------------------------------------------------------ */

/* Free-flow time in ms: length[dm] * 360 / speed[km/h], rounded half up, at least 1, at most 2^26. */
uint32_t orc_free_flow_ms(uint32_t length_dm, uint32_t speed_kmh)
{
    uint64_t num = (uint64_t)length_dm * 360u + speed_kmh / 2u;
    uint64_t ff = num / speed_kmh;
    if (ff < 1)
        ff = 1;
    if (ff > ORC_TIME_CLAMP)
        ff = ORC_TIME_CLAMP;
    return (uint32_t)ff;
}

/* Jam capacity in vehicles: lanes * length / 7.5 m, at least 1. */
uint32_t orc_capacity(uint32_t lanes, uint32_t length_dm)
{
    uint64_t c = (uint64_t)lanes * length_dm / 75u;
    return c < 1 ? 1u : (uint32_t)c;
}

/* Congested travel time: ff * cap / max(cap - n, max(1, cap/20)), floor, at most 2^26 ms. */
uint32_t orc_edge_time_ms(uint32_t ff_ms, uint32_t cap, uint32_t n)
{
    uint64_t floor_den = cap / 20u;
    if (floor_den < 1)
        floor_den = 1;
    uint64_t den = floor_den;
    if (n < cap && (uint64_t)(cap - n) > floor_den)
        den = cap - n;
    uint64_t t = (uint64_t)ff_ms * cap / den;
    return t > ORC_TIME_CLAMP ? ORC_TIME_CLAMP : (uint32_t)t;
}

/* Queue discharge delay at a signalised head: n * h_sat / lanes, floor, at most 2^26 ms; else 0. */
uint32_t orc_queue_delay_ms(uint32_t n, uint32_t h_sat_ms, uint32_t lanes, int head_signalised)
{
    if (!head_signalised)
        return 0;
    uint64_t d = (uint64_t)n * h_sat_ms / lanes;
    return d > ORC_TIME_CLAMP ? ORC_TIME_CLAMP : (uint32_t)d;
}

/* ------------------------------------------------------------------------------------------------ */
/* Preemptive signal rule (Fig. 3 signal block; Calc_Dens / Comp_Thres, Sec. 4.2 and Algorithm 2).    */
/* Produces the order in which the phases receive green in the next cycle; green                      */
/* durations stay as programmed.                                                                       */
/* ------------------------------------------------------------------------------------------------ */
void orc_phase_order(uint32_t n_phases, const uint64_t *Q, const uint64_t *Th, const uint32_t *red_ms,
                     uint32_t T_max, uint8_t *order)
{
    int used[ORC_MAX_PHASES] = {0};
    uint32_t n = 0;
    int any_over = 0, any_starved = 0;
    for (uint32_t p = 0; p < n_phases; ++p) {
        if (Q[p] > Th[p])
            any_over = 1;
        if (red_ms[p] > T_max)
            any_starved = 1;
    }
    if (any_over) {
        /* (1) every phase whose queue exceeds its threshold, longest queue first */
        for (;;) {
            int best = -1;
            for (uint32_t p = 0; p < n_phases; ++p)
                if (!used[p] && Q[p] > Th[p] && (best < 0 || Q[p] > Q[best]))
                    best = (int)p;
            if (best < 0)
                break;
            used[best] = 1;
            order[n++] = (uint8_t)best;
        }
    } else if (any_starved) {
        /* (2) every phase red for longer than T_max, longest wait first */
        for (;;) {
            int best = -1;
            for (uint32_t p = 0; p < n_phases; ++p)
                if (!used[p] && red_ms[p] > T_max && (best < 0 || red_ms[p] > red_ms[best]))
                    best = (int)p;
            if (best < 0)
                break;
            used[best] = 1;
            order[n++] = (uint8_t)best;
        }
    } else {
        /* (3) the phase with the longest queue goes first, if any queue is non-empty */
        int best = -1;
        for (uint32_t p = 0; p < n_phases; ++p)
            if (Q[p] > 0 && (best < 0 || Q[p] > Q[best]))
                best = (int)p;
        if (best >= 0) {
            used[best] = 1;
            order[n++] = (uint8_t)best;
        }
    }
    /* the rest keep the default order; phases with an empty queue are skipped to the end */
    for (uint32_t p = 0; p < n_phases; ++p)
        if (!used[p] && Q[p] > 0) {
            used[p] = 1;
            order[n++] = (uint8_t)p;
        }
    for (uint32_t p = 0; p < n_phases; ++p)
        if (!used[p]) {
            used[p] = 1;
            order[n++] = (uint8_t)p;
        }
    for (uint32_t i = n_phases; i < ORC_MAX_PHASES; ++i)
        order[i] = (uint8_t)i;
}

static uint32_t hsat_of(const orc_params *prm)
{
    return (prm && prm->h_sat_ms) ? prm->h_sat_ms : ORC_DEFAULT_HSAT;
}

/* Per-node phase order from the current densities (dt = 0: densities and red accumulators fixed). */
int orc_queue_preempt(const orc_net *g, const orc_params *prm, uint8_t *order_out)
{
    (void)prm;
    uint32_t N = g->n_nodes;
    uint64_t *Q = calloc((size_t)N * ORC_MAX_PHASES + 1, sizeof(uint64_t));
    uint64_t *capsum = calloc((size_t)N * ORC_MAX_PHASES + 1, sizeof(uint64_t));
    if (!Q || !capsum) {
        free(Q);
        free(capsum);
        return ORC_ERR_OOM;
    }
    /* Calc_Dens: vehicles queued on the approaches of each phase, one pass over all roads */
    for (uint32_t u = 0; u < N; ++u)
        for (uint32_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) {
            uint32_t v = g->col[e];
            if (g->n_phases[v] == 0)
                continue;
            uint32_t p = g->edge_phase[e];
            if (p >= g->n_phases[v]) {
                free(Q);
                free(capsum);
                return ORC_ERR_INVALID;
            }
            Q[(size_t)v * ORC_MAX_PHASES + p] += g->vehicles[e];
            capsum[(size_t)v * ORC_MAX_PHASES + p] += orc_capacity(g->lanes[e], g->length_dm[e]);
        }
    for (uint32_t v = 0; v < N; ++v) {
        uint32_t P = g->n_phases[v];
        uint8_t *ord = order_out + (size_t)v * ORC_MAX_PHASES;
        if (P == 0) {
            for (uint32_t i = 0; i < ORC_MAX_PHASES; ++i)
                ord[i] = (uint8_t)i;
            continue;
        }
        uint64_t Th[ORC_MAX_PHASES] = {0};
        uint32_t red[ORC_MAX_PHASES] = {0};
        for (uint32_t p = 0; p < P; ++p) {
            Th[p] = capsum[(size_t)v * ORC_MAX_PHASES + p] * 3u / 4u; /* Comp_Thres: 3/4 of approach storage */
            red[p] = g->red_ms ? g->red_ms[(size_t)v * ORC_MAX_PHASES + p] : 0u;
        }
        orc_phase_order(P, Q + (size_t)v * ORC_MAX_PHASES, Th, red, g->cycle_ms[v], ord);
    }
    free(Q);
    free(capsum);
    return ORC_OK;
}

/* Wait at a signal: arrival at time arr (ms), phase windows laid out from the node's offset in the
 * given phase order. Zero inside the approach phase's green window, otherwise the time until it starts. */
uint32_t orc_signal_wait_ms(uint64_t arr_ms, uint32_t cycle, uint32_t offset, const uint32_t *green,
                            const uint8_t *order, uint32_t n_phases, uint32_t phase)
{
    uint64_t start = 0;
    for (uint32_t i = 0; i < n_phases; ++i) {
        if (order[i] == phase)
            break;
        start += green[order[i]];
    }
    uint64_t c = (arr_ms % cycle + cycle - (offset % cycle)) % cycle; /* position in the cycle */
    if (c >= start && c < start + green[phase])
        return 0;
    return (uint32_t)((start + cycle - c) % cycle);
}

/* kappa = floor(360 * 2^16 / v_max): ms per dm at the network's top speed, Q16.16. */
uint64_t orc_kappa(uint32_t v_max_kmh)
{
    return ((uint64_t)360u << 16) / v_max_kmh;
}

/* Calc_Dist: lower bound on the remaining time from (x,y) to the destination. */
uint32_t orc_heuristic_ms(int32_t x, int32_t y, int32_t xd, int32_t yd, uint64_t kappa)
{
    int64_t dx = (int64_t)x - xd, dy = (int64_t)y - yd;
    uint64_t d2 = (uint64_t)(dx * dx) + (uint64_t)(dy * dy);
    uint64_t h = (orc_isqrt64(d2) * kappa) >> 16;
    return h > ORC_H_CLAMP ? ORC_H_CLAMP : (uint32_t)h;
}

/* ------------------------------------------------------------------------------------------------ */
/* Next-node rule (Fig. 3's node selection; Algorithm 2): roulette over tau^alpha * eta^beta.   */
/* ------------------------------------------------------------------------------------------------ */
static float pow_int(float x, uint32_t k)
{
    if (k == 0)
        return 1.0f;
    float p = x;
    for (uint32_t i = 1; i < k; ++i)
        p = p * x;
    return p;
}

/* The pheromone factor of a score as binary32: tau * 2^-32, or its reciprocal (one rounded division)
 * when less pheromone is preferred. tau >= 1, so both are normal and at most 2^32. */
float orc_tau_factor(uint64_t tau, uint32_t flags)
{
    float tf = (float)tau * 0x1p-32f;
    return (flags & ORC_FLAG_REPULSIVE) ? 1.0f / tf : tf;
}

/* s = f^alpha * (1 / c)^beta with f = orc_tau_factor(tau), each step one rounded binary32 operation.
 * f^alpha saturates at the largest finite binary32 (f < 2^32 overflows from alpha = 5 on), so every
 * score is finite and eta^beta <= 1 keeps the product finite too. */
float orc_score_f(uint64_t tau, uint32_t alpha, uint32_t c_ms, uint32_t beta, uint32_t flags)
{
    float p = pow_int(orc_tau_factor(tau, flags), alpha);
    if (p > FLT_MAX)
        p = FLT_MAX;
    float eta = 1.0f / (float)c_ms;
    return p * pow_int(eta, beta);
}

float orc_score(uint64_t tau, uint32_t alpha, uint32_t c_ms, uint32_t beta)
{
    return orc_score_f(tau, alpha, c_ms, beta, 0u);
}

/* ------------------------------------------------------------------------------------------------ */
/* Non-integer alpha / beta: the score as 2^L, L = alpha*log2(f) - beta*log2(c), with a binary32       */
/* log2 and exp2 of our own. Both are fixed sequences of single rounded binary32 operations.          */
/* ------------------------------------------------------------------------------------------------ */
/* Series coefficients, each the nearest binary32 to its exact value:
 * 1/3, 1/5, 1/7, 1/9 (atanh), 2/ln 2, and ln(2)^k / k! for k = 1..8 (Taylor series of 2^f). */
static const float LOG_C3 = 0x1.555556p-2f, LOG_C5 = 0x1.99999ap-3f, LOG_C7 = 0x1.24924ap-3f,
                   LOG_C9 = 0x1.c71c72p-4f, LOG_K = 0x1.715476p+1f;
static const float EXP_C[9] = {1.0f,          0x1.62e430p-1f, 0x1.ebfbe0p-3f, 0x1.c6b08ep-5f, 0x1.3b2ab6p-7f,
                               0x1.5d87fep-10f, 0x1.430912p-13f, 0x1.ffcbfcp-17f, 0x1.62c022p-20f};

void orc_frac_constants(float out[14])
{
    out[0] = LOG_C3;
    out[1] = LOG_C5;
    out[2] = LOG_C7;
    out[3] = LOG_C9;
    out[4] = LOG_K;
    for (int k = 0; k < 9; ++k)
        out[5 + k] = EXP_C[k];
}

static float bits_to_float(uint32_t b)
{
    float f;
    memcpy(&f, &b, 4);
    return f;
}

static uint32_t float_to_bits(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

/* log2 x for a positive normal binary32 x. Range reduction as in Cody & Waite (Software Manual for
 * the Elementary Functions, 1980): x = 2^e * m with m in (1/sqrt 2, sqrt 2]; then
 * ln m = 2 atanh(t), t = (m - 1) / (m + 1), |t| <= 0.1716, by the atanh series through t^9:
 * log2 m = t * (2/ln 2) * (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9) (truncation below 2^-28 relative). */
float orc_log2(float x)
{
    uint32_t b = float_to_bits(x);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x7FFFFFu) | 0x3F800000u;
    if (mb > 0x3FB504F3u) { /* m above sqrt 2 (rounded down): use m/2 */
        mb -= 0x00800000u;
        e += 1;
    }
    float m = bits_to_float(mb);
    float t = (m - 1.0f) / (m + 1.0f);
    float t2 = t * t;
    float p = LOG_C9;
    p = p * t2 + LOG_C7;
    p = p * t2 + LOG_C5;
    p = p * t2 + LOG_C3;
    p = p * t2 + 1.0f;
    float r = (t * LOG_K) * p;
    return (float)e + r;
}

/* 2^L in binary32: FLT_MAX for L >= 128 (saturation, as for integer exponents), 0 below -150;
 * otherwise n = floor(L), f = L - n in [0, 1) (exact), 2^f by its Taylor series through f^8 in Horner
 * form (truncation below 2^-26 relative), capped below 2, times 2^n in two exact power-of-two steps
 * (the second rounds only into the subnormal range). */
float orc_exp2(float L)
{
    if (!(L < 128.0f))
        return FLT_MAX;
    if (L < -150.0f)
        return 0.0f;
    float n = floorf(L);
    float f = L - n;
    float p = EXP_C[8];
    for (int k = 7; k >= 0; --k)
        p = p * f + EXP_C[k];
    const float below2 = 0x1.fffffep0f;
    if (p > below2)
        p = below2;
    int ni = (int)n;
    int n1 = ni >= 0 ? ni / 2 : -((-ni + 1) / 2); /* floor(ni / 2) */
    int n2 = ni - n1;
    float s1 = bits_to_float((uint32_t)(n1 + 127) << 23), s2 = bits_to_float((uint32_t)(n2 + 127) << 23);
    return (p * s1) * s2;
}

/* Score for non-integer exponents: 2^(alpha*log2 f - beta*log2 c), f = orc_tau_factor(tau), c as
 * binary32 (rounded to nearest above 2^24). Equals f^alpha * (1/c)^beta up to the error bound pinned
 * in the tests. */
float orc_score_frac(uint64_t tau, float alpha, uint32_t c_ms, float beta, uint32_t flags)
{
    float A = alpha * orc_log2(orc_tau_factor(tau, flags));
    float B = beta * orc_log2((float)c_ms);
    return orc_exp2(A - B);
}

/* Integer roulette weights: w_i = max(1, floor(s_i * 2^(22 - E))) with E = floor(log2(max s));
 * all ones when every score is zero. Every weight is below 2^23, so the running sums of up to 512
 * candidates fit in 32 bits. */
void orc_quantize(uint32_t n, const float *s, uint64_t *w)
{
    float m = 0.0f;
    for (uint32_t i = 0; i < n; ++i)
        if (s[i] > m)
            m = s[i];
    if (m == 0.0f) {
        for (uint32_t i = 0; i < n; ++i)
            w[i] = 1;
        return;
    }
    int e2;
    (void)frexp((double)m, &e2); /* m = f * 2^e2, f in [0.5, 1) */
    int E = e2 - 1;
    for (uint32_t i = 0; i < n; ++i) {
        double v = floor(ldexp((double)s[i], 22 - E));
        uint64_t q = (uint64_t)v;
        w[i] = q < 1 ? 1 : q;
    }
}

/* First index whose running weight sum exceeds r = floor(rnd * S / 2^64). */
uint32_t orc_roulette_pick(uint32_t n, const uint64_t *w, uint64_t rnd)
{
    uint64_t S = 0;
    for (uint32_t i = 0; i < n; ++i)
        S += w[i];
    uint64_t r = (uint64_t)(((unsigned __int128)rnd * S) >> 64);
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) {
        acc += w[i];
        if (acc > r)
            return i;
    }
    return n - 1; /* unreachable: r < S */
}

/* rho_fix = round(rho * 2^32), ties to even, computed in double. */
uint64_t orc_rho_fix(float rho)
{
    return (uint64_t)nearbyint(ldexp((double)rho, 32));
}

/* Evap_Pher on one road: tau - floor(tau * rho_fix / 2^32). */
uint64_t orc_evaporate(uint64_t tau, uint64_t rho_fix)
{
    return tau - (uint64_t)(((unsigned __int128)tau * rho_fix) >> 32);
}

/* ------------------------------------------------------------------------------------------------ */
/* Exact Calc_Dist (Algorithm 2 computes the distance to the destination over the routes of the      */
/* graph): h(v) = the least sum of congested travel times over the roads of a path from v to dst,      */
/* by Dijkstra's algorithm from dst over the reversed roads; nodes that cannot reach dst, and sums     */
/* beyond it, take the clamp 2^28. Waits are not included, so h never exceeds the remaining time.      */
/* ------------------------------------------------------------------------------------------------ */
int orc_exact_heuristic(const orc_net *g, const uint32_t *tt, uint32_t dst, uint32_t *h)
{
    uint32_t N = g->n_nodes, E = g->n_edges;
    uint32_t *rptr = calloc((size_t)N + 1, sizeof(uint32_t)), *redge = malloc(sizeof(uint32_t) * (E + 1));
    uint32_t *tail = malloc(sizeof(uint32_t) * (E + 1));
    uint64_t *dist = malloc(sizeof(uint64_t) * (N + 1));
    uint8_t *done = calloc((size_t)N + 1, 1);
    if (!rptr || !redge || !tail || !dist || !done) {
        free(rptr);
        free(redge);
        free(tail);
        free(dist);
        free(done);
        return ORC_ERR_OOM;
    }
    /* roads grouped by head: the reversed graph */
    for (uint32_t u = 0; u < N; ++u)
        for (uint32_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) {
            tail[e] = u;
            rptr[g->col[e] + 1]++;
        }
    for (uint32_t v = 0; v < N; ++v)
        rptr[v + 1] += rptr[v];
    {
        uint32_t *fill = malloc(sizeof(uint32_t) * (N + 1));
        if (!fill) {
            free(rptr);
            free(redge);
            free(tail);
            free(dist);
            free(done);
            return ORC_ERR_OOM;
        }
        memcpy(fill, rptr, sizeof(uint32_t) * N);
        for (uint32_t e = 0; e < E; ++e)
            redge[fill[g->col[e]]++] = e;
        free(fill);
    }
    for (uint32_t v = 0; v < N; ++v)
        dist[v] = UINT64_MAX;
    dist[dst] = 0;
    /* Dijkstra with a binary min-heap of (distance, node) entries and lazy deletion: an entry whose
     * distance is above the node's current one is stale and skipped */
    size_t cap = (size_t)E + 2, n_heap = 0;
    uint64_t *hk = malloc(sizeof(uint64_t) * cap);
    uint32_t *hv = malloc(sizeof(uint32_t) * cap);
    if (!hk || !hv) {
        free(hk);
        free(hv);
        free(rptr);
        free(redge);
        free(tail);
        free(dist);
        free(done);
        return ORC_ERR_OOM;
    }
#define HEAP_SWAP(a, b)                                                                                  \
    do {                                                                                                 \
        uint64_t tk = hk[a];                                                                             \
        uint32_t tv = hv[a];                                                                             \
        hk[a] = hk[b];                                                                                   \
        hv[a] = hv[b];                                                                                   \
        hk[b] = tk;                                                                                      \
        hv[b] = tv;                                                                                      \
    } while (0)
    hk[0] = 0;
    hv[0] = dst;
    n_heap = 1;
    while (n_heap > 0) {
        uint64_t d = hk[0];
        uint32_t u = hv[0];
        hk[0] = hk[--n_heap]; /* pop the root, sift the last entry down */
        hv[0] = hv[n_heap];
        for (size_t i = 0;;) {
            size_t l = 2 * i + 1, r = l + 1, m = i;
            if (l < n_heap && hk[l] < hk[m])
                m = l;
            if (r < n_heap && hk[r] < hk[m])
                m = r;
            if (m == i)
                break;
            HEAP_SWAP(i, m);
            i = m;
        }
        if (done[u] || d > dist[u])
            continue;
        done[u] = 1;
        for (uint32_t i = rptr[u]; i < rptr[u + 1]; ++i) {
            uint32_t e = redge[i], v = tail[e];
            uint64_t nd = dist[u] + tt[e];
            if (nd < dist[v]) {
                dist[v] = nd;
                size_t j = n_heap++; /* push, sift up (each road pushes at most once: cap = E + 2) */
                hk[j] = nd;
                hv[j] = v;
                while (j > 0 && hk[(j - 1) / 2] > hk[j]) {
                    HEAP_SWAP(j, (j - 1) / 2);
                    j = (j - 1) / 2;
                }
            }
        }
    }
#undef HEAP_SWAP
    free(hk);
    free(hv);
    for (uint32_t v = 0; v < N; ++v)
        h[v] = dist[v] > ORC_H_CLAMP ? ORC_H_CLAMP : (uint32_t)dist[v];
    free(rptr);
    free(redge);
    free(tail);
    free(dist);
    free(done);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Solve state                                                                                          */
/* ------------------------------------------------------------------------------------------------ */
typedef struct {
    const orc_net *g;
    uint32_t max_steps, thr, t_dep, flags;
    uint32_t *ff, *cap, *tt, *qd, *h;
    uint8_t *order; /* N*8 */
    uint8_t *visited;
    uint32_t *cand;
    float *score;
    uint32_t *waitv;
    uint64_t *w;
    uint32_t *wait_at; /* wait taken at each position of the current route */
} orc_state;

static void state_free(orc_state *S)
{
    free(S->ff);
    free(S->cap);
    free(S->tt);
    free(S->qd);
    free(S->h);
    free(S->order);
    free(S->visited);
    free(S->cand);
    free(S->score);
    free(S->waitv);
    free(S->w);
    free(S->wait_at);
}

static int state_init(orc_state *S, const orc_net *g, const orc_params *prm, uint32_t dst)
{
    memset(S, 0, sizeof *S);
    S->g = g;
    uint32_t N = g->n_nodes, E = g->n_edges;
    uint32_t maxdeg = 0;
    for (uint32_t v = 0; v < N; ++v)
        if (g->row_ptr[v + 1] - g->row_ptr[v] > maxdeg)
            maxdeg = g->row_ptr[v + 1] - g->row_ptr[v];
    S->ff = malloc(sizeof(uint32_t) * (E + 1));
    S->cap = malloc(sizeof(uint32_t) * (E + 1));
    S->tt = malloc(sizeof(uint32_t) * (E + 1));
    S->qd = malloc(sizeof(uint32_t) * (E + 1));
    S->h = malloc(sizeof(uint32_t) * (N + 1));
    S->order = malloc((size_t)N * ORC_MAX_PHASES + 1);
    S->visited = malloc(N + 1);
    S->cand = malloc(sizeof(uint32_t) * (maxdeg + 1));
    S->score = malloc(sizeof(float) * (maxdeg + 1));
    S->waitv = malloc(sizeof(uint32_t) * (maxdeg + 1));
    S->w = malloc(sizeof(uint64_t) * (maxdeg + 1));
    if (!S->ff || !S->cap || !S->tt || !S->qd || !S->h || !S->order || !S->visited || !S->cand || !S->score ||
        !S->waitv || !S->w) {
        state_free(S);
        return ORC_ERR_OOM;
    }
    uint32_t hsat = hsat_of(prm);
    uint32_t vmax = 1;
    for (uint32_t u = 0; u < N; ++u)
        for (uint32_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) {
            uint32_t v = g->col[e];
            S->ff[e] = orc_free_flow_ms(g->length_dm[e], g->speed_kmh[e]);
            S->cap[e] = orc_capacity(g->lanes[e], g->length_dm[e]);
            S->tt[e] = orc_edge_time_ms(S->ff[e], S->cap[e], g->vehicles[e]);
            S->qd[e] = orc_queue_delay_ms(g->vehicles[e], hsat, g->lanes[e], g->n_phases[v] > 0);
            if (g->speed_kmh[e] > vmax)
                vmax = g->speed_kmh[e];
        }
    uint64_t kappa = orc_kappa(vmax);
    if (prm && (prm->flags & ORC_FLAG_EXACT_H)) {
        int hr = orc_exact_heuristic(g, S->tt, dst, S->h);
        if (hr != ORC_OK) {
            state_free(S);
            return hr;
        }
    } else {
        for (uint32_t v = 0; v < N; ++v)
            S->h[v] = orc_heuristic_ms(g->x_dm[v], g->y_dm[v], g->x_dm[dst], g->y_dm[dst], kappa);
    }
    int rc = orc_queue_preempt(g, prm, S->order);
    if (rc != ORC_OK) {
        state_free(S);
        return rc;
    }
    /* a depth-first walk reaches every node it can reach, and returns, within 2(N-1) moves */
    uint64_t two_n = 2ull * (N - 1u);
    uint32_t def_steps = two_n < 4096u ? (uint32_t)two_n : 4096u;
    S->max_steps = (prm && prm->max_steps) ? prm->max_steps : def_steps;
    S->thr = prm ? prm->thr_permille : ORC_THR_OFF;
    S->t_dep = prm ? prm->t_dep_ms : 0u;
    S->flags = prm ? prm->flags : 0u;
    /* a route never has more roads than moves were made (nor, being a simple path, more than N - 1) */
    S->wait_at = malloc(sizeof(uint32_t) * ((size_t)S->max_steps + 1));
    if (!S->wait_at) {
        state_free(S);
        return ORC_ERR_OOM;
    }
    return ORC_OK;
}

/* One ant of iteration `it` (Fig. 3 body for one vehicle, with the roulette next-node rule). The ant keeps
 * a visited set, so its route is a simple path. At a node where no road leads to an unvisited node it
 * steps back along its route to the previous node: that node's elapsed time and wait come back, the node
 * it left stays visited, and the step back counts as a move. It fails when it is back at src with no
 * road left, after max_steps moves, or when its elapsed time exceeds 2^30 ms. The draw of a forward move
 * is keyed by the move's index. A road's cost is the time it adds over the remaining lower bound:
 * c = tt + wait + h(v) - h(u), at least 1 ms. Writes the route's roads to route_edges; returns the ant
 * status. */
static int walk(orc_state *S, const orc_query *q, uint32_t alpha, uint32_t beta, int frac, const uint64_t *tau,
                uint32_t it, uint32_t ant, uint32_t *route_edges, uint32_t *len_out, uint32_t *moves_out,
                uint32_t *T_out, uint32_t *W_out)
{
    const orc_net *g = S->g;
    memset(S->visited, 0, g->n_nodes);
    uint32_t u = q->src, moves = 0, len = 0;
    uint64_t t = 0, W = 0;
    int status;
    S->visited[u] = 1;
    for (;;) {
        if (u == q->dst) {
            status = ANT_SUCCESS;
            break;
        }
        if (moves == S->max_steps) {
            status = ANT_STEP_CAP;
            break;
        }
        /* Adj_Neigh: roads out of u whose head has not been visited, in CSR order */
        uint32_t n = 0;
        for (uint32_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e)
            if (!S->visited[g->col[e]])
                S->cand[n++] = e;
        /* congestion threshold (Fig. 3's test of N_t): congested roads drop out unless all are */
        if (S->thr != ORC_THR_OFF && n > 0) {
            uint32_t n_ok = 0;
            for (uint32_t i = 0; i < n; ++i) {
                uint32_t e = S->cand[i];
                if ((uint64_t)g->vehicles[e] * 1000u <= (uint64_t)S->thr * S->cap[e])
                    n_ok++;
            }
            if (n_ok > 0 && n_ok < n) {
                uint32_t m = 0;
                for (uint32_t i = 0; i < n; ++i) {
                    uint32_t e = S->cand[i];
                    if ((uint64_t)g->vehicles[e] * 1000u <= (uint64_t)S->thr * S->cap[e])
                        S->cand[m++] = e;
                }
                n = m;
            }
        }
        if (n == 0) {
            if (len == 0) {
                status = ANT_DEAD_END;
                break;
            }
            /* dead end: back to the previous node of the route, with the time and wait it had there */
            len--;
            uint32_t e = route_edges[len];
            t -= (uint64_t)S->tt[e] + S->wait_at[len];
            W -= S->wait_at[len];
            u = len ? g->col[route_edges[len - 1]] : q->src;
            moves++;
            continue;
        }
        /* Eval_Rout: travel time, signal wait + queue delay at the head, change of the remaining bound */
        for (uint32_t i = 0; i < n; ++i) {
            uint32_t e = S->cand[i], v = g->col[e];
            uint32_t w = 0;
            if (v != q->dst && g->n_phases[v] > 0) {
                uint64_t arr = (uint64_t)S->t_dep + t + S->tt[e];
                w = orc_signal_wait_ms(arr, g->cycle_ms[v], g->offset_ms[v], g->green_ms + (size_t)v * ORC_MAX_PHASES,
                                       S->order + (size_t)v * ORC_MAX_PHASES, g->n_phases[v], g->edge_phase[e]) +
                    S->qd[e];
            }
            int64_t cost = (int64_t)S->tt[e] + w + S->h[v] - S->h[u];
            uint32_t c = cost < 1 ? 1u : (uint32_t)cost;
            S->waitv[i] = w;
            S->score[i] = frac ? orc_score_frac(tau[e], q->alpha, c, q->beta, S->flags)
                               : orc_score_f(tau[e], alpha, c, beta, S->flags);
        }
        orc_quantize(n, S->score, S->w);
        uint32_t pick = orc_roulette_pick(n, S->w, draw64(q->seed, it, ant, moves, 0));
        uint32_t e = S->cand[pick];
        /* position update */
        t += (uint64_t)S->tt[e] + S->waitv[pick];
        W += S->waitv[pick];
        u = g->col[e];
        S->visited[u] = 1;
        S->wait_at[len] = S->waitv[pick];
        route_edges[len++] = e;
        moves++;
        if (t > ORC_T_CAP) {
            status = ANT_TIME_CAP;
            break;
        }
    }
    *len_out = len;
    *moves_out = moves;
    *T_out = (uint32_t)t;
    *W_out = (uint32_t)W;
    return status;
}

/* alpha, beta in [0, 8]; integers take the repeated-multiplication score, anything else the 2^L score. */
static int query_ok(const orc_net *g, const orc_query *q, uint32_t *alpha, uint32_t *beta, int *frac)
{
    if (q->src >= g->n_nodes || q->dst >= g->n_nodes || q->n_ants == 0 || q->n_iter == 0)
        return ORC_ERR_INVALID;
    if ((uint64_t)q->n_ants * q->n_iter > 0xFFFFFFFFull)
        return ORC_ERR_INVALID;
    if (!(q->alpha >= 0.0f && q->alpha <= 8.0f && q->beta >= 0.0f && q->beta <= 8.0f))
        return ORC_ERR_UNSUPPORTED;
    if (!(q->rho >= 0.0f && q->rho < 1.0f))
        return ORC_ERR_INVALID;
    *frac = floorf(q->alpha) != q->alpha || floorf(q->beta) != q->beta;
    *alpha = (uint32_t)q->alpha;
    *beta = (uint32_t)q->beta;
    return ORC_OK;
}

/* Derived per-road and per-node quantities, for tests. Any output may be NULL. */
int orc_prepare(const orc_net *g, const orc_params *prm, uint32_t dst, uint32_t *ff, uint32_t *cap, uint32_t *tt,
                uint32_t *qd, uint32_t *h, uint8_t *order)
{
    orc_state S;
    int rc = state_init(&S, g, prm, dst);
    if (rc != ORC_OK)
        return rc;
    size_t E = g->n_edges, N = g->n_nodes;
    if (ff)
        memcpy(ff, S.ff, E * 4);
    if (cap)
        memcpy(cap, S.cap, E * 4);
    if (tt)
        memcpy(tt, S.tt, E * 4);
    if (qd)
        memcpy(qd, S.qd, E * 4);
    if (h)
        memcpy(h, S.h, N * 4);
    if (order)
        memcpy(order, S.order, N * ORC_MAX_PHASES);
    state_free(&S);
    return ORC_OK;
}

/* One ant walk against a given pheromone table (for hand-worked tests): route_edges receives the route
 * (*len roads), *moves counts its forward moves and steps back. */
int orc_walk_one(const orc_net *g, const orc_params *prm, const orc_query *q, const uint64_t *tau, uint32_t it,
                 uint32_t ant, uint32_t *route_edges, uint32_t *len, uint32_t *moves, uint32_t *T, uint32_t *W)
{
    uint32_t alpha, beta;
    int frac;
    int rc = query_ok(g, q, &alpha, &beta, &frac);
    if (rc != ORC_OK)
        return -rc;
    orc_state S;
    rc = state_init(&S, g, prm, q->dst);
    if (rc != ORC_OK)
        return -rc;
    int st = walk(&S, q, alpha, beta, frac, tau, it, ant, route_edges, len, moves, T, W);
    state_free(&S);
    return st;
}

/* Initial pheromone (Algorithm 2): 1.0 in Q32.32, or with the random flag
 * 0.5 + u/2^32 where u is word 0 of Philox(counter = (road, 0, 0, 1), key = seed). */
void orc_init_tau(uint32_t E, uint64_t seed, uint32_t flags, uint64_t *tau)
{
    for (uint32_t e = 0; e < E; ++e) {
        if (flags & ORC_FLAG_RANDOM_TAU) {
            uint32_t c[4] = {e, 0, 0, 1}, k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, o[4];
            orc_philox4x32_10(c, k, o);
            tau[e] = ((uint64_t)1 << 31) + o[0];
        } else {
            tau[e] = (uint64_t)1 << 32;
        }
    }
}

/*
 * The full colony for one origin-destination query (Algorithms 1-2 with Fig. 3's per-vehicle body):
 *   for it in 0..I-1: every ant walks on the pheromone of the previous iteration; successful ants
 *   deposit floor(max(h(src),1) * 2^32 / T) on each road of their route; then every road evaporates
 *   and receives its deposits; then the per-intersection phase order is recomputed.
 * The paper's own variant, by flags: ORC_FLAG_UNIT_DEPOSIT makes each deposit exactly 1.0 (Ph_road++);
 * ORC_FLAG_EVAP_UNUSED adds the deposits first and then evaporates only the roads that received none
 * (Updt_Pher before Evap_Pher, which decrements unused roads); ORC_FLAG_REPULSIVE acts in the walk.
 * route_nodes receives the best route (min T, then lowest (iteration, ant)) as node ids, src first.
 * tau_out (E entries, may be NULL) receives the final pheromone. ant_log (may be NULL) receives per
 * (iteration, ant) {status | roads in the route << 8, moves, T, W}; res->ant_steps counts every move of
 * every ant, forward or back.
 */
int orc_solve(const orc_net *g, const orc_params *prm, const orc_query *q, uint32_t *route_nodes, uint32_t route_cap,
              uint64_t *tau_out, uint32_t *ant_log, orc_result *res)
{
    memset(res, 0, sizeof *res);
    uint32_t alpha, beta;
    int frac;
    int rc = query_ok(g, q, &alpha, &beta, &frac);
    if (rc != ORC_OK) {
        res->status = rc;
        return rc;
    }
    if (prm && prm->t_dep_ms >= ORC_T_CAP) {
        res->status = ORC_ERR_INVALID;
        return ORC_ERR_INVALID;
    }
    uint32_t E = g->n_edges;
    uint64_t *tau = malloc(sizeof(uint64_t) * (E + 1));
    uint64_t *D = malloc(sizeof(uint64_t) * (E + 1));
    orc_state S;
    int init_rc = state_init(&S, g, prm, q->dst);
    size_t route_max = init_rc == ORC_OK ? (size_t)S.max_steps + 1 : 1;
    uint32_t *route = malloc(sizeof(uint32_t) * route_max);
    uint32_t *best_route = malloc(sizeof(uint32_t) * route_max);
    if (init_rc == ORC_OK && (!tau || !D || !route || !best_route))
        state_free(&S);
    if (!tau || !D || !route || !best_route || init_rc != ORC_OK) {
        free(tau);
        free(D);
        free(route);
        free(best_route);
        res->status = ORC_ERR_OOM;
        return ORC_ERR_OOM;
    }
    orc_init_tau(E, q->seed, prm ? prm->flags : 0u, tau);

    uint64_t best_key = UINT64_MAX;
    uint32_t best_len = 0, best_W = 0;
    if (q->src == q->dst) {
        best_key = 0;
    } else {
        uint64_t rho_fix = orc_rho_fix(q->rho);
        uint64_t dep_num = (uint64_t)(S.h[q->src] > 0 ? S.h[q->src] : 1u) << 32;
        int unit = (S.flags & ORC_FLAG_UNIT_DEPOSIT) != 0;
        for (uint32_t it = 0; it < q->n_iter; ++it) {
            memset(D, 0, sizeof(uint64_t) * E);
            for (uint32_t k = 0; k < q->n_ants; ++k) {
                uint32_t steps, moves, T, W;
                int st = walk(&S, q, alpha, beta, frac, tau, it, k, route, &steps, &moves, &T, &W);
                res->ant_steps += moves;
                if (ant_log) {
                    uint32_t *l = ant_log + 4 * ((size_t)it * q->n_ants + k);
                    l[0] = (uint32_t)st | (steps << 8);
                    l[1] = moves;
                    l[2] = T;
                    l[3] = W;
                }
                if (st != ANT_SUCCESS)
                    continue;
                res->n_success++;
                /* Updt_Pher: every successful ant deposits on the roads it used */
                uint64_t delta = unit ? (uint64_t)1 << 32 : dep_num / T;
                for (uint32_t i = 0; i < steps; ++i)
                    D[route[i]] += delta;
                uint64_t key = ((uint64_t)T << 32) | ((uint64_t)it * q->n_ants + k);
                if (key < best_key) {
                    best_key = key;
                    best_len = steps;
                    best_W = W;
                    memcpy(best_route, route, sizeof(uint32_t) * steps);
                }
            }
            if (S.flags & ORC_FLAG_EVAP_UNUSED) {
                /* Updt_Pher, then Evap_Pher on the roads no successful ant used */
                for (uint32_t e = 0; e < E; ++e)
                    tau[e] += D[e];
                for (uint32_t e = 0; e < E; ++e)
                    if (D[e] == 0)
                        tau[e] = orc_evaporate(tau[e], rho_fix);
            } else {
                /* Evap_Pher + deposit */
                for (uint32_t e = 0; e < E; ++e)
                    tau[e] = orc_evaporate(tau[e], rho_fix) + D[e];
            }
            /* per-iteration queue/preemption update (densities are fixed during a solve) */
            orc_queue_preempt(g, prm, S.order);
        }
    }
    if (tau_out)
        memcpy(tau_out, tau, sizeof(uint64_t) * E);
    if (best_key == UINT64_MAX) {
        res->status = ORC_ERR_NO_ROUTE;
    } else {
        res->status = ORC_OK;
        res->travel_ms = best_key >> 32;
        res->wait_ms = best_W;
        res->route_len = best_len + 1;
        if (q->src != q->dst) {
            uint32_t low = (uint32_t)best_key;
            res->best_iter = low / q->n_ants;
            res->best_ant = low % q->n_ants;
        }
        if (route_cap < best_len + 1) {
            res->status = ORC_ERR_BUFFER;
        } else {
            route_nodes[0] = q->src;
            for (uint32_t i = 0; i < best_len; ++i)
                route_nodes[i + 1] = g->col[best_route[i]];
        }
    }
    state_free(&S);
    free(tau);
    free(D);
    free(route);
    free(best_route);
    return res->status;
}

/* ------------------------------------------------------------------------------------------------ */
/* Serving tick: the queue / preemption update with dt > 0 (Fig. 3 signal block; Calc_Dens and        */
/* Comp_Thres of Sec. 4.2 applied to vehicles that move). One step of length dt at clock t_now:        */
/*   green phase of each signalised node from its current phase order (every approach is served at an  */
/*   unsignalised node); each served road discharges min(n, c) vehicles, c = lanes*(t_now+dt)/h_sat -   */
/*   lanes*t_now/h_sat (saturation flow counted on the whole clock, so no fraction is lost); a node's    */
/*   discharge K is split over its d out-roads, K/d each and one more for the first K mod d in CSR      */
/*   order (vehicles leave the network at nodes without out-roads); red-time accumulators: 0 for the    */
/*   green phase, + dt (saturating at 2^32-1) for other phases with a queue, 0 for empty phases (queues */
/*   counted before the discharge); then the phase order is recomputed from the new state. Vehicle      */
/*   counts are 32-bit and wrap like unsigned arithmetic.                                                */
/* ------------------------------------------------------------------------------------------------ */
static uint32_t green_phase_at(uint64_t t, uint32_t cycle, uint32_t offset, const uint32_t *green,
                               const uint8_t *order, uint32_t P)
{
    uint64_t c = (t % cycle + cycle - (offset % cycle)) % cycle;
    uint64_t start = 0;
    for (uint32_t i = 0; i < P; ++i) {
        uint32_t p = order[i];
        if (c >= start && c < start + green[p])
            return p;
        start += green[p];
    }
    return order[P - 1]; /* unreachable: greens cover the cycle */
}

int orc_tick(const orc_net *g, const orc_params *prm, uint64_t t_now, uint32_t dt, const uint8_t *order,
             uint32_t *veh_out, uint32_t *red_out, uint8_t *order_out)
{
    uint32_t N = g->n_nodes, E = g->n_edges, hsat = hsat_of(prm);
    uint32_t *leave = calloc((size_t)E + 1, sizeof(uint32_t));
    uint64_t *K = calloc((size_t)N + 1, sizeof(uint64_t));
    uint64_t *Q = calloc((size_t)N * ORC_MAX_PHASES + 1, sizeof(uint64_t));
    uint32_t *gph = malloc(sizeof(uint32_t) * ((size_t)N + 1));
    if (!leave || !K || !Q || !gph) {
        free(leave);
        free(K);
        free(Q);
        free(gph);
        return ORC_ERR_OOM;
    }
    for (uint32_t v = 0; v < N; ++v)
        gph[v] = g->n_phases[v] ? green_phase_at(t_now, g->cycle_ms[v], g->offset_ms[v],
                                                 g->green_ms + (size_t)v * ORC_MAX_PHASES,
                                                 order + (size_t)v * ORC_MAX_PHASES, g->n_phases[v])
                                : 0xFFFFFFFFu;
    /* queues before the discharge, and the discharge of every served road */
    for (uint32_t u = 0; u < N; ++u)
        for (uint32_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) {
            uint32_t v = g->col[e], n = g->vehicles[e];
            if (g->n_phases[v])
                Q[(size_t)v * ORC_MAX_PHASES + g->edge_phase[e]] += n;
            if (g->n_phases[v] == 0 || g->edge_phase[e] == gph[v]) {
                /* saturation flow lanes/h_sat, counted on the whole clock so no fraction is lost */
                uint64_t cap = (uint64_t)g->lanes[e] * (t_now + dt) / hsat - (uint64_t)g->lanes[e] * t_now / hsat;
                leave[e] = (uint32_t)(n < cap ? n : cap);
                K[v] += leave[e];
            }
        }
    /* the discharge of each node goes to its out-roads */
    for (uint32_t u = 0; u < N; ++u) {
        uint32_t b = g->row_ptr[u], d = g->row_ptr[u + 1] - b;
        for (uint32_t j = 0; j < d; ++j) {
            uint32_t e = b + j;
            uint64_t in = K[u] / d + (j < K[u] % d ? 1u : 0u);
            veh_out[e] = (uint32_t)(g->vehicles[e] - leave[e] + in);
        }
    }
    for (uint32_t v = 0; v < N; ++v)
        for (uint32_t p = 0; p < ORC_MAX_PHASES; ++p) {
            size_t i = (size_t)v * ORC_MAX_PHASES + p;
            uint32_t r = g->red_ms ? g->red_ms[i] : 0u;
            if (g->n_phases[v] == 0 || p >= g->n_phases[v] || p == gph[v] || Q[i] == 0)
                red_out[i] = 0;
            else
                red_out[i] = r > 0xFFFFFFFFu - dt ? 0xFFFFFFFFu : r + dt;
        }
    /* the new phase order from the new vehicles and red times */
    orc_net g2 = *g;
    g2.vehicles = veh_out;
    g2.red_ms = red_out;
    int rc = orc_queue_preempt(&g2, prm, order_out);
    free(leave);
    free(K);
    free(Q);
    free(gph);
    return rc;
}

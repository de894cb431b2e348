// Device-side data layout and arithmetic of the sm_103a MACO-P colony.
//
// Everything here is integer or single IEEE binary32 operations with explicit round-to-nearest
// intrinsics (__fmul_rn, __fdiv_rn, __ull2float_rn ...), so results do not depend on FMA contraction,
// thread mapping or the order in which warps finish.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmacop.h"

namespace gmp {

constexpr uint32_t kMaxPhases = 8;
constexpr uint32_t kTimeClamp = 1u << 26;  // edge travel times and queue delays saturate at 2^26 ms
constexpr uint32_t kHClamp = 1u << 28;     // heuristic lower bound saturates at 2^28 ms
constexpr uint32_t kTCap = 1u << 30;       // an ant whose elapsed time exceeds 2^30 ms fails
constexpr uint32_t kHsatDefault = 2000;    // saturation headway per lane, ms
constexpr uint32_t kThrOff = 0xFFFFFFFFu;
constexpr uint64_t kNoKey = ~0ull;

enum : uint32_t { kAntSuccess = 0, kAntDeadEnd = 1, kAntStepCap = 2, kAntTimeCap = 3 };

// Per-road record read by the construction kernel: everything one candidate needs in two 16-byte
// loads. The first half (head, its CSR row start, congested time, queue delay and the congestion flag)
// follows the densities; the second half (the head's out-degree, and its signal cycle, this approach's
// green window and a reciprocal for reducing arrival times modulo the cycle) follows the phase order.
struct __align__(16) EdgeRec {
    uint32_t head;    // v
    uint32_t vbeg;    // first road out of v
    uint32_t tt;      // congested travel time, ms
    uint32_t qd_fl;   // queue discharge delay at v, ms (bits 0-30; 0 when v is unsignalised) |
                      // road over the congestion threshold (bit 31)
    uint32_t cyc_deg; // cycle of v's signal (bits 0-23; 0 = unsignalised) | out-degree of v (bits 24-31)
    uint32_t gbeg;    // start of this approach's green window, (offset + start in phase order) mod cycle
    uint32_t glen;    // green time of this approach's phase
    uint32_t cmagic;  // floor((2^32 - 1) / cycle), 0 when unsignalised
};
static_assert(sizeof(EdgeRec) == 32, "EdgeRec layout");
constexpr uint32_t kCycleMask = 0xFFFFFFu;  // cycles are below 2^24 ms
constexpr uint32_t kQdMask = 0x7FFFFFFFu;

// One colony of a batch, as the kernels read it.
struct __align__(16) DevQuery {
    uint32_t src, dst, n_ants, n_iter;
    uint32_t alpha, beta, ant_base, active;  // active == 0 when src == dst (answered without ants); with
                                             // kQueryFracExp set, alpha and beta hold binary32 bits
    uint64_t rho_fix;                        // round(rho * 2^32)
    uint64_t seed;
    int32_t xd, yd;                          // destination coordinates
    uint64_t log_base;                       // first entry of this query in the ant log
};
static_assert(sizeof(DevQuery) == 64, "DevQuery layout");

// Per-colony running state.
struct __align__(16) QueryState {
    unsigned long long best_key;  // (T << 32) | (iteration * n_ants + ant); kNoKey = none yet
    unsigned long long dep_num;   // max(h(src), 1) << 32: a successful ant deposits dep_num / T per road;
                                  // 0 under GMP_FLAG_UNIT_DEPOSIT (every deposit is 1.0)
    unsigned long long steps;     // roads taken by all ants
    unsigned long long nsucc;     // successful walks
    uint32_t best_len;            // roads in the best route
    uint32_t best_W;              // waits along the best route
    uint32_t h_src;               // h(src): the remaining bound where every walk starts
    uint32_t pad;
    // sparse pheromone layout: every road without a deposit so far holds the same value, the baseline
    unsigned long long base_tau;  // baseline tau of the current iteration (Q32.32)
    uint32_t base_tf;             // its binary32 image (bits)
    uint32_t n_touched;           // roads with a deposit so far (entries of the colony's touched list)
};
static_assert(sizeof(QueryState) == 64, "QueryState layout");

// Result row copied back to the host.
struct __align__(16) DevResult {
    uint64_t travel_ms, wait_ms, ant_steps, n_success;
    uint32_t route_len, best_iter, best_ant;
    int32_t status;
};
static_assert(sizeof(DevResult) == 48, "DevResult layout");

// ------------------------------------------------------------------------------------------------
// Counter-based generator: Philox4x32-10 (Salmon et al., SC'11), ten rounds of two 32x32 -> 64-bit
// products and a word permutation, key bumped by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// floor(sqrt(n)) for n < 2^58: a binary32 estimate (n from its two 32-bit halves, the hardware's
// approximate square root) corrected to the exact integer root. The root is below 2^29, so the checks
// are single 32 x 32 -> 64-bit products. The estimate is within about r / 2^22 of the root r: under two
// units, so at most two turns of the loops, for distances below 2^22 dm (about 420 km).
__device__ __forceinline__ uint32_t isqrt_u64(uint64_t n) {
    const float f = __fmaf_rn(__uint2float_rn((uint32_t)(n >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)n));
    float s;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(f));
    uint32_t r = __float2uint_rz(s);
    while ((uint64_t)r * r > n) --r;
    while ((uint64_t)(r + 1u) * (r + 1u) <= n) ++r;
    return r;
}

// Calc_Dist: admissible remaining-time bound, floor(isqrt(dx^2 + dy^2) * kappa / 2^16), kappa =
// floor(360 * 2^16 / v_max) ms per dm in Q16.16. Coordinates lie within +-2^27 dm (checked when the graph
// is loaded), so the differences fit in 32 bits and their squares are single wide products.
__device__ __forceinline__ uint32_t heuristic_ms(int32_t x, int32_t y, int32_t xd, int32_t yd, uint32_t kappa) {
    const int32_t dx = x - xd, dy = y - yd;
    const uint64_t d = isqrt_u64((uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy));
    const uint64_t h = (d * kappa) >> 16;
    return h > kHClamp ? kHClamp : (uint32_t)h;
}

// x mod d for x < 2^32 and 1 <= d <= 2^24, with m = floor((2^32 - 1) / d): the quotient estimate
// floor(x * m / 2^32) is exact or one too small, so one conditional subtraction finishes it.
__device__ __forceinline__ uint32_t mod_magic(uint32_t x, uint32_t d, uint32_t m) {
    const uint32_t q = __umulhi(x, m);
    const uint32_t r = x - q * d;
    return r >= d ? r - d : r;
}

// Signal wait for a vehicle reaching the stop line at absolute time arr: the approach is green during
// [gbeg, gbeg + glen) modulo the cycle; otherwise it waits for the next start of that window.
__device__ __forceinline__ uint32_t signal_wait(uint32_t arr, uint32_t cycle, uint32_t cmagic, uint32_t gbeg,
                                                uint32_t glen) {
    const uint32_t x = mod_magic(arr, cycle, cmagic);
    const uint32_t c = x >= gbeg ? x - gbeg : x + (cycle - gbeg);
    return c < glen ? 0u : cycle - c;
}

// x^k by repeated multiplication left to right (x^0 = 1); k is uniform across the lanes of an ant.
__device__ __forceinline__ float pow_int(float x, uint32_t k) {
    if (k == 0) return 1.0f;
    float p = x;
    for (uint32_t i = 1; i < k; ++i) p = __fmul_rn(p, x);
    return p;
}

// Pheromone as a binary32 value: the Q32.32 integer rounded to nearest, scaled exactly by 2^-32.
__device__ __forceinline__ float tau_float(uint64_t tau) { return __fmul_rn(__ull2float_rn(tau), 0x1p-32f); }

// The binary32 word a candidate's score reads for pheromone tau (bits): tau_float(tau), or under
// GMP_FLAG_REPULSIVE its reciprocal rounded to nearest, so that less pheromone scores higher (Sec. 4.1).
// tau >= 1, so both are normal, at most 2^32 and never 0 (0 marks a road at the sparse baseline).
__device__ __forceinline__ uint32_t tau_word(uint64_t tau, uint32_t flags) {
    const float tf = tau_float(tau);
    return __float_as_uint((flags & GMP_FLAG_REPULSIVE) ? __frcp_rn(tf) : tf);
}

// One iteration's pheromone update of a road holding tau with deposits d (Evap_Pher, Updt_Pher):
// tau - floor(tau * rho_fix / 2^32) + d; under GMP_FLAG_EVAP_UNUSED a road with deposits keeps tau + d
// and only a road without any evaporates.
__device__ __forceinline__ uint64_t tau_next(uint64_t t, uint64_t rho_fix, uint64_t d, uint32_t flags) {
    const uint64_t lo = t * rho_fix, hi = __umul64hi(t, rho_fix);
    const uint64_t ev = t - ((hi << 32) | (lo >> 32));
    return ((flags & GMP_FLAG_EVAP_UNUSED) && d) ? t + d : ev + d;
}

// Deposit of a successful ant of elapsed time T on each road of its route (Updt_Pher): dep_num / T, or
// exactly 1.0 when dep_num is 0 (GMP_FLAG_UNIT_DEPOSIT, the paper's Ph_road++).
__device__ __forceinline__ unsigned long long ant_deposit(unsigned long long dep_num, uint32_t T) {
    return dep_num ? dep_num / T : (1ull << 32);
}

// 1 / c rounded to nearest for 1 <= c <= 2^29 (results are never subnormal): the hardware reciprocal
// estimate corrected once with fused multiply-adds (Markstein, IBM J. Res. Dev. 34(1), 1990: the
// residual 1 - c*y is exact in an FMA, and one FMA correction of a faithful estimate is correctly
// rounded). Equal to __frcp_rn(c) for every float in [1, 2^29], checked exhaustively on the GPU.
__device__ __forceinline__ float rcp_rn(float c) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(c));
    const float r = __fmaf_rn(-c, y, 1.0f);
    return __fmaf_rn(r, y, y);
}

// c as binary32 rounded to nearest for c < 2^29, on the floating-point pipe: both halves of
// c = 64*floor(c/64) + (c mod 64) are exact (2^23 + x - 2^23 for x < 2^23) and one FMA rounds their
// exact sum once. Equal to __uint2float_rn(c) for every c < 2^29 (checked exhaustively on the GPU).
__device__ __forceinline__ float u32_to_f32_rn(uint32_t c) {
    const float hi = __fsub_rn(__uint_as_float(0x4B000000u | (c >> 6)), 8388608.0f);
    const float lo = __fsub_rn(__uint_as_float(0x4B000000u | (c & 63u)), 8388608.0f);
    return __fmaf_rn(hi, 64.0f, lo);
}

// ------------------------------------------------------------------------------------------------
// Non-integer alpha / beta: the score as 2^L, L = alpha*log2(f) - beta*log2(c), from a binary32 log2
// and exp2 of our own (single rounded operations, no FMA contraction).
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kQueryFracExp = 2u;  // DevQuery::active bit: alpha and beta are binary32 bits

// Series coefficients, each the binary32 nearest its exact value: 1/3, 1/5, 1/7, 1/9 and 2/ln 2 for
// the atanh series of log2; ln(2)^k / k! for k = 1..8 for the Taylor series of 2^f.
constexpr float kLogC3 = 0x1.555556p-2f, kLogC5 = 0x1.99999ap-3f, kLogC7 = 0x1.24924ap-3f, kLogC9 = 0x1.c71c72p-4f,
                kLogK = 0x1.715476p+1f;
constexpr float kExpC1 = 0x1.62e430p-1f, kExpC2 = 0x1.ebfbe0p-3f, kExpC3 = 0x1.c6b08ep-5f, kExpC4 = 0x1.3b2ab6p-7f,
                kExpC5 = 0x1.5d87fep-10f, kExpC6 = 0x1.430912p-13f, kExpC7 = 0x1.ffcbfcp-17f,
                kExpC8 = 0x1.62c022p-20f;

// log2 x for a positive normal x: x = 2^e * m with m in (1/sqrt 2, sqrt 2] (the range reduction of
// Cody & Waite, Software Manual for the Elementary Functions, 1980), then ln m = 2 atanh(t),
// t = (m - 1) / (m + 1), |t| <= 0.1716, by the atanh series through t^9 (truncation below 2^-28).
__device__ __forceinline__ float log2_cw(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x7FFFFFu) | 0x3F800000u;
    if (mb > 0x3FB504F3u) {  // m above sqrt 2 (rounded down): use m / 2
        mb -= 0x00800000u;
        ++e;
    }
    const float m = __uint_as_float(mb);
    const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float p = kLogC9;
    p = __fadd_rn(__fmul_rn(p, t2), kLogC7);
    p = __fadd_rn(__fmul_rn(p, t2), kLogC5);
    p = __fadd_rn(__fmul_rn(p, t2), kLogC3);
    p = __fadd_rn(__fmul_rn(p, t2), 1.0f);
    return __fadd_rn(__int2float_rn(e), __fmul_rn(__fmul_rn(t, kLogK), p));
}

// 2^L: the largest finite binary32 for L >= 128 (saturation, as for integer exponents), 0 below -150;
// else n = floor(L), f = L - n in [0, 1) (exact), 2^f by its Taylor series through f^8 (truncation
// below 2^-26) capped below 2, scaled by 2^n in two exact power-of-two steps (the second rounds only
// into the subnormal range).
__device__ __forceinline__ float exp2_sat(float L) {
    if (!(L < 128.0f)) return 3.40282347e38f;
    if (L < -150.0f) return 0.0f;
    const float n = floorf(L);
    const float f = __fsub_rn(L, n);
    float p = kExpC8;
    p = __fadd_rn(__fmul_rn(p, f), kExpC7);
    p = __fadd_rn(__fmul_rn(p, f), kExpC6);
    p = __fadd_rn(__fmul_rn(p, f), kExpC5);
    p = __fadd_rn(__fmul_rn(p, f), kExpC4);
    p = __fadd_rn(__fmul_rn(p, f), kExpC3);
    p = __fadd_rn(__fmul_rn(p, f), kExpC2);
    p = __fadd_rn(__fmul_rn(p, f), kExpC1);
    p = __fadd_rn(__fmul_rn(p, f), 1.0f);
    p = fminf(p, 0x1.fffffep0f);
    const int ni = (int)n;
    const int n1 = ni >> 1, n2 = ni - n1;  // floor(n / 2): both in [-75, 64]
    return __fmul_rn(__fmul_rn(p, __uint_as_float((uint32_t)(n1 + 127) << 23)),
                     __uint_as_float((uint32_t)(n2 + 127) << 23));
}

// Score for non-integer exponents (alpha, beta in [0, 8] as floats): 2^(alpha log2 tf - beta log2 c).
__device__ __forceinline__ float score_frac(float tf, float alpha, uint32_t c, float beta) {
    const float A = __fmul_rn(alpha, log2_cw(tf));
    const float B = __fmul_rn(beta, log2_cw(u32_to_f32_rn(c)));
    return exp2_sat(__fsub_rn(A, B));
}

// Next-node desirability from the pheromone word tf (tau_word): tf^alpha * (1 / c)^beta, c = travel +
// wait + remaining bound (ms), 1 <= c < 2^29. tf < 2^32, so tf^alpha can overflow from alpha = 5 on:
// it saturates at the largest finite binary32, and eta^beta <= 1 keeps every score finite (the roulette
// weights need a finite maximum). The alpha = 1, beta = 2 case performs the same roundings in the same
// order without loops (it cannot overflow).
__device__ __forceinline__ float score_f(float tf, uint32_t alpha, uint32_t c, uint32_t beta) {
    const float eta = rcp_rn(u32_to_f32_rn(c));
    if (alpha == 1u && beta == 2u) return __fmul_rn(tf, __fmul_rn(eta, eta));
    return __fmul_rn(fminf(pow_int(tf, alpha), 3.40282347e38f), pow_int(eta, beta));
}

// The score of a colony: integer exponents by score_f, others (frac) by score_frac with alpha and beta
// as binary32 bits.
// Cost of a road in the score: the time it adds over the remaining lower bound, from the sum
// tt + wait + h(head) (below 2^29) and h of the node the ant stands on; at least 1 ms.
__device__ __forceinline__ uint32_t reduced_cost(uint32_t c_through, uint32_t h_here) {
    return c_through > h_here ? c_through - h_here : 1u;
}

__device__ __forceinline__ float score_q(float tf, uint32_t alpha, uint32_t c, uint32_t beta, bool frac) {
    if (frac) return score_frac(tf, __uint_as_float(alpha), c, __uint_as_float(beta));
    return score_f(tf, alpha, c, beta);
}

// The roulette's index r = floor(rnd * S / 2^64) for a 64-bit draw and S < 2^32, from two 32x32 -> 64
// products: floor((hi*S*2^32 + lo*S) / 2^64) = (hi*S + floor(lo*S / 2^32)) >> 32 (the dropped fraction
// cannot carry across a multiple of 2^32).
__device__ __forceinline__ uint32_t draw_index(unsigned long long rnd, uint32_t S) {
    const uint32_t lo = (uint32_t)rnd, hi = (uint32_t)(rnd >> 32);
    const unsigned long long a = (unsigned long long)hi * S, b = ((unsigned long long)lo * S) >> 32;
    return (uint32_t)((a + b) >> 32);
}

// A non-negative binary32 bit pattern as (M, X) with value = M * 2^(X - 150): M in [2^23, 2^24) for
// every non-zero value, M = 0 for zero. A subnormal is first scaled by 2^64 (exact) to read its
// exponent. No branches.
__device__ __forceinline__ void norm_f32(uint32_t bits, uint32_t& M, int& X) {
    const uint32_t e = bits >> 23;
    const uint32_t b2 = __float_as_uint(__fmul_rn(__uint_as_float(bits), 0x1p64f));
    const uint32_t src = e ? bits : b2;
    M = bits ? ((src & 0x7FFFFFu) | 0x800000u) : 0u;
    X = e ? (int)e : (int)(b2 >> 23) - 64;
}

// Integer roulette weight relative to the largest score m (given as its exponent Xm and whether it is
// zero): floor(s * 2^(22 - floor(log2 m))) = M_s >> (X_m - X_s + 1), at least 1; all ones when m == 0.
// Below 2^23, so running sums of up to 512 weights fit in 32 bits. No branches.
__device__ __forceinline__ uint32_t roulette_weight_x(uint32_t sbits, int Xm, bool mzero) {
    uint32_t Ms;
    int Xs;
    norm_f32(sbits, Ms, Xs);
    const int d = max(1, min(Xm - Xs + 1, 31));  // masked-out slots may carry any value: keep the shift defined
    const uint32_t w = Ms >> d;
    return (mzero || w == 0u) ? 1u : w;
}

__device__ __forceinline__ uint32_t roulette_weight(uint32_t sbits, uint32_t mbits) {
    uint32_t Mm;
    int Xm;
    norm_f32(mbits, Mm, Xm);
    return roulette_weight_x(sbits, Xm, mbits == 0u);
}

// The same weights in binary32 arithmetic. For a step whose largest score m has E = floor(log2 m),
// scale = (2^k1, 2^k2) with k1 + k2 = 22 - E, both factors normal. v = s * 2^k1 * 2^k2 < 2^23 is exact:
// multiplying by a power of two is exact unless the result leaves the normal range, and any result
// that does so (a shrinking first factor) makes v below 1, where the weight is 1 anyway. floor(v) is
// then one addition of 2^23 rounded toward zero.
struct WeightScale {
    float s1, s2;
    bool mzero;
};

__device__ __forceinline__ WeightScale weight_scale(uint32_t mbits) {
    uint32_t Mm;
    int Xm;
    norm_f32(mbits, Mm, Xm);
    const int k = 22 - (Xm - 127);  // 22 - E, in [-105, 171]
    const int k1 = k >> 1, k2 = k - k1;
    WeightScale w;
    w.s1 = __uint_as_float((uint32_t)(k1 + 127) << 23);
    w.s2 = __uint_as_float((uint32_t)(k2 + 127) << 23);
    w.mzero = mbits == 0u;
    return w;
}

__device__ __forceinline__ uint32_t roulette_weight_f(uint32_t sbits, const WeightScale& sc) {
    const float v = __fmul_rn(__fmul_rn(__uint_as_float(sbits), sc.s1), sc.s2);
    const uint32_t w = __float_as_uint(__fadd_rz(v, 8388608.0f)) - 0x4B000000u;  // floor(v), v < 2^23
    return (sc.mzero || w == 0u) ? 1u : w;
}

// floor(a * b / d) for 32-bit operands and d >= 1: a 32-bit division when the product fits 32 bits.
__device__ __forceinline__ uint64_t mul_div_u32(uint32_t a, uint32_t b, uint32_t d) {
    const uint64_t p = (uint64_t)a * b;
    return (p >> 32) == 0 ? (uint64_t)((uint32_t)p / d) : p / d;
}

// Congested travel time ff * cap / max(cap - n, max(1, cap / 20)), saturating at 2^26 ms.
__device__ __forceinline__ uint32_t edge_time_ms(uint32_t ff, uint32_t cap, uint32_t n) {
    uint32_t fl = cap / 20u;
    if (fl < 1u) fl = 1u;
    const uint32_t den = (n < cap && cap - n > fl) ? cap - n : fl;
    const uint64_t t = mul_div_u32(ff, cap, den);
    return t > kTimeClamp ? kTimeClamp : (uint32_t)t;
}

}  // namespace gmp

// Device-side data layout and arithmetic of the sm_103a MACO-P colony.
//
// Everything here is integer or single IEEE binary32 operations with explicit round-to-nearest
// intrinsics (__fmul_rn, __fdiv_rn, __ull2float_rn ...), so results do not depend on FMA contraction,
// thread mapping or the order in which warps finish.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gmp {

constexpr uint32_t kMaxPhases = 8;
constexpr uint32_t kTimeClamp = 1u << 26;  // edge travel times and queue delays saturate at 2^26 ms
constexpr uint32_t kHClamp = 1u << 28;     // heuristic lower bound saturates at 2^28 ms
constexpr uint32_t kTCap = 1u << 30;       // an ant whose elapsed time exceeds 2^30 ms fails
constexpr uint32_t kHsatDefault = 2000;    // saturation headway per lane, ms
constexpr uint32_t kThrOff = 0xFFFFFFFFu;
constexpr uint64_t kNoKey = ~0ull;

enum : uint32_t { kAntSuccess = 0, kAntDeadEnd = 1, kAntStepCap = 2, kAntTimeCap = 3 };

// Per-road record read by the construction kernel: everything one candidate needs in three 16-byte
// loads (the head's CSR row, congested time, queue delay, the head signal's green window for this
// approach and a reciprocal for reducing arrival times modulo the cycle). Rebuilt whenever densities,
// signals or the phase order change.
struct __align__(16) EdgeRec {
    uint32_t head;   // v
    uint32_t vbeg;   // first road out of v
    uint32_t vend;   // one past the last road out of v
    uint32_t tt;     // congested travel time, ms
    uint32_t qd;     // queue discharge delay at v (0 when v is unsignalised), ms
    uint32_t cycle;  // cycle of v's signal, 0 = unsignalised
    uint32_t gbeg;   // start of this approach's green window, (offset + start in phase order) mod cycle
    uint32_t glen;   // green time of this approach's phase
    unsigned long long cmagic;  // floor((2^64 - 1) / cycle), 0 when unsignalised
    uint32_t flags;  // bit 0: road over the congestion threshold
    uint32_t pad;
};
static_assert(sizeof(EdgeRec) == 48, "EdgeRec layout");

// One colony of a batch, as the kernels read it.
struct __align__(16) DevQuery {
    uint32_t src, dst, n_ants, n_iter;
    uint32_t alpha, beta, ant_base, active;  // active == 0 when src == dst (answered without ants)
    uint64_t rho_fix;                        // round(rho * 2^32)
    uint64_t seed;
    int32_t xd, yd;                          // destination coordinates
    uint64_t log_base;                       // first entry of this query in the ant log
};
static_assert(sizeof(DevQuery) == 64, "DevQuery layout");

// Per-colony running state.
struct __align__(16) QueryState {
    unsigned long long best_key;  // (T << 32) | (iteration * n_ants + ant); kNoKey = none yet
    unsigned long long dep_num;   // max(h(src), 1) << 32: a successful ant deposits dep_num / T per road
    unsigned long long steps;     // roads taken by all ants
    unsigned long long nsucc;     // successful walks
    uint32_t best_len;            // roads in the best route
    uint32_t best_W;              // waits along the best route
    uint32_t pad[2];
};
static_assert(sizeof(QueryState) == 48, "QueryState layout");

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

// floor(sqrt(n)) for n < 2^58: a binary32 estimate corrected to the exact integer root.
__device__ __forceinline__ uint64_t isqrt_u64(uint64_t n) {
    uint64_t r = (uint64_t)__fsqrt_rn(__ull2float_rn(n));
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}

// Calc_Dist: admissible remaining-time bound, floor(isqrt(dx^2 + dy^2) * kappa / 2^16), kappa =
// floor(360 * 2^16 / v_max) ms per dm in Q16.16.
__device__ __forceinline__ uint32_t heuristic_ms(int32_t x, int32_t y, int32_t xd, int32_t yd, uint32_t kappa) {
    const int64_t dx = (int64_t)x - xd, dy = (int64_t)y - yd;
    const uint64_t d = isqrt_u64((uint64_t)(dx * dx) + (uint64_t)(dy * dy));
    const uint64_t h = (d * kappa) >> 16;
    return h > kHClamp ? kHClamp : (uint32_t)h;
}

// x mod d for x < 2^32 and 1 <= d <= 2^24, with m = floor((2^64 - 1) / d): the quotient estimate
// floor(x * m / 2^64) is exact or one too small, so one conditional subtraction finishes it.
__device__ __forceinline__ uint32_t mod_magic(uint32_t x, uint32_t d, unsigned long long m) {
    const uint32_t q = (uint32_t)__umul64hi((unsigned long long)x, m);
    const uint32_t r = x - q * d;
    return r >= d ? r - d : r;
}

// Signal wait for a vehicle reaching the stop line at absolute time arr: the approach is green during
// [gbeg, gbeg + glen) modulo the cycle; otherwise it waits for the next start of that window.
__device__ __forceinline__ uint32_t signal_wait(uint32_t arr, uint32_t cycle, unsigned long long cmagic,
                                                uint32_t gbeg, uint32_t glen) {
    const uint32_t x = mod_magic(arr, cycle, cmagic);
    const uint32_t c = x >= gbeg ? x - gbeg : x + (cycle - gbeg);
    return c < glen ? 0u : cycle - c;
}

// x^k for 0 <= k <= 8 by repeated multiplication left to right (x^0 = 1), without branches.
__device__ __forceinline__ float pow_int(float x, uint32_t k) {
    float p = k ? x : 1.0f;
#pragma unroll
    for (uint32_t i = 2; i <= 8; ++i) {
        const float y = __fmul_rn(p, x);
        p = i <= k ? y : p;
    }
    return p;
}

// Next-node desirability: (tau / 2^32)^alpha * (1 / c)^beta, c = travel + wait + remaining bound (ms).
// __frcp_rn(c) is 1/c rounded to nearest, the same value as the division 1.0f / c.
__device__ __forceinline__ float score(uint64_t tau, uint32_t alpha, uint32_t c, uint32_t beta) {
    const float tf = __fmul_rn(__ull2float_rn(tau), 0x1p-32f);
    const float eta = __frcp_rn(__uint2float_rn(c));
    return __fmul_rn(pow_int(tf, alpha), pow_int(eta, beta));
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// A non-negative binary32 value as mant * 2^(ex - 150) with mant in [2^23, 2^24) (subnormals
// normalised); zero gives mant = 0.
__device__ __forceinline__ void split_f32(uint32_t bits, uint32_t& mant, int& ex) {
    const uint32_t e = bits >> 23, m = bits & 0x7FFFFFu;
    if (e) {
        mant = m | 0x800000u;
        ex = (int)e;
    } else if (m) {
        const int sh = __clz(m) - 8;
        mant = m << sh;
        ex = 1 - sh;
    } else {
        mant = 0;
        ex = -1024;
    }
}

// Integer roulette weight relative to the largest score: floor(s * 2^(30 - floor(log2 max))) at least 1.
__device__ __forceinline__ uint32_t roulette_weight(uint32_t sbits, uint32_t mmant, int mex) {
    if (mmant == 0) return 1u;  // every score is zero: uniform choice
    uint32_t mant;
    int ex;
    split_f32(sbits, mant, ex);
    const int d = mex - ex;
    const uint32_t w = d >= 31 ? 0u : (mant << 7) >> d;
    return w ? w : 1u;
}

// Congested travel time ff * cap / max(cap - n, max(1, cap / 20)), saturating at 2^26 ms.
__device__ __forceinline__ uint32_t edge_time_ms(uint32_t ff, uint32_t cap, uint32_t n) {
    uint32_t fl = cap / 20u;
    if (fl < 1u) fl = 1u;
    const uint32_t den = (n < cap && cap - n > fl) ? cap - n : fl;
    const uint64_t t = (uint64_t)ff * cap / den;
    return t > kTimeClamp ? kTimeClamp : (uint32_t)t;
}

}  // namespace gmp

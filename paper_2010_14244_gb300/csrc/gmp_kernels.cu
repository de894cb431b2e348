// sm_103a kernels of the MACO-P route colony (Jindal & Bedi, GMACO-P, Sec. 4.2, Algorithm 2).
//
//   k_edge_static     road free-flow time and jam capacity                         (graph load)
//   k_edge_dynamic    congested travel time, queue delay, threshold flag per road   (Calc_Dens inputs)
//   k_queue_preempt   per-intersection phase order by the preemptive rule         (Calc_Dens, Comp_Thres)
//   k_init_batch      initial pheromone, per-colony state                          (Algorithm 2 step 3)
//   k_construct<G,K>  ant walks: Adj_Neigh, next-node roulette, Eval_Rout, position update, deposits
//   k_evaporate       Evap_Pher fused with the deposits of Updt_Pher
//   k_best_copy       best-route tracking
//   k_finalize        best route as node ids + counters
#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp_device.cuh"
#include "gmp_internal.h"

namespace gmp {

// ------------------------------------------------------------------------------------------------
// Road attributes
// ------------------------------------------------------------------------------------------------
__global__ void k_edge_static(uint32_t E, const uint32_t* __restrict__ len, const uint16_t* __restrict__ speed,
                              const uint8_t* __restrict__ lanes, uint32_t* __restrict__ ff, uint32_t* __restrict__ cap) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const uint64_t L = len[e], v = speed[e];
    uint64_t f = (L * 360u + v / 2u) / v;  // length / speed in ms, rounded half up
    f = f < 1u ? 1u : (f > kTimeClamp ? kTimeClamp : f);
    ff[e] = (uint32_t)f;
    const uint64_t c = (uint64_t)lanes[e] * L / 75u;  // one vehicle per 7.5 m of lane
    cap[e] = c < 1u ? 1u : (uint32_t)c;
}

__global__ void k_edge_dynamic(uint32_t E, const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                               const uint32_t* __restrict__ ff, const uint32_t* __restrict__ cap,
                               const uint8_t* __restrict__ lanes, const uint32_t* __restrict__ veh,
                               const uint8_t* __restrict__ nph, uint32_t h_sat, uint32_t thr,
                               EdgeRec* __restrict__ rec) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const uint32_t v = col[e], n = veh[e], c = cap[e];
    EdgeRec& r = rec[e];
    r.head = v;
    r.vbeg = row_ptr[v];
    r.vend = row_ptr[v + 1];
    r.tt = edge_time_ms(ff[e], c, n);
    uint32_t qd = 0;
    if (nph[v] > 0) {
        const uint64_t d = (uint64_t)n * h_sat / lanes[e];
        qd = d > kTimeClamp ? kTimeClamp : (uint32_t)d;
    }
    r.qd = qd;
    r.flags = (thr != kThrOff && (uint64_t)n * 1000u > (uint64_t)thr * c) ? 1u : 0u;
    r.pad = 0;
}

// ------------------------------------------------------------------------------------------------
// Preemptive phase order, one thread per intersection. Queues and storage per phase come from the
// road's in-edges (reverse CSR). Order: (1) phases whose queue exceeds 3/4 of their storage, longest
// first; else (2) phases red for longer than a cycle, longest first; else (3) the longest non-empty
// queue. Then the remaining non-empty phases, then the empty ones, each in default (index) order.
// Every in-edge's record then gets its approach's green window under that order.
// ------------------------------------------------------------------------------------------------
__global__ void k_queue_preempt(uint32_t N, const uint32_t* __restrict__ in_ptr, const uint32_t* __restrict__ in_edge,
                                const uint8_t* __restrict__ nph, const uint32_t* __restrict__ cycle,
                                const uint32_t* __restrict__ offset, const uint32_t* __restrict__ green,
                                const uint8_t* __restrict__ ephase, const uint32_t* __restrict__ veh,
                                const uint32_t* __restrict__ cap, const uint32_t* __restrict__ red,
                                uint8_t* __restrict__ order, EdgeRec* __restrict__ rec) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const uint32_t P = nph[v], ib = in_ptr[v], ie = in_ptr[v + 1];
    uint8_t ord[kMaxPhases];
    if (P == 0) {
        for (uint32_t i = 0; i < kMaxPhases; ++i) order[(size_t)v * kMaxPhases + i] = (uint8_t)i;
        for (uint32_t i = ib; i < ie; ++i) {
            EdgeRec& r = rec[in_edge[i]];
            r.cycle = 0;
            r.gbeg = 0;
            r.glen = 0;
            r.cmagic = 0;
        }
        return;
    }
    uint64_t Q[kMaxPhases], S[kMaxPhases];
    for (uint32_t p = 0; p < kMaxPhases; ++p) Q[p] = S[p] = 0;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t e = in_edge[i];
        const uint32_t p = ephase[e] & (kMaxPhases - 1);
        Q[p] += veh[e];
        S[p] += cap[e];
    }
    const uint32_t cy = cycle[v];
    uint32_t over = 0, starved = 0, nonempty = 0;
    uint32_t rd[kMaxPhases];
    for (uint32_t p = 0; p < P; ++p) {
        rd[p] = red[(size_t)v * kMaxPhases + p];
        if (Q[p] > S[p] * 3u / 4u) over |= 1u << p;
        if (rd[p] > cy) starved |= 1u << p;
        if (Q[p] > 0) nonempty |= 1u << p;
    }
    uint32_t used = 0, n = 0;
    if (over) {
        while (over & ~used) {
            int best = -1;
            for (uint32_t p = 0; p < P; ++p)
                if ((over & ~used) >> p & 1u)
                    if (best < 0 || Q[p] > Q[best]) best = (int)p;
            used |= 1u << best;
            ord[n++] = (uint8_t)best;
        }
    } else if (starved) {
        while (starved & ~used) {
            int best = -1;
            for (uint32_t p = 0; p < P; ++p)
                if ((starved & ~used) >> p & 1u)
                    if (best < 0 || rd[p] > rd[best]) best = (int)p;
            used |= 1u << best;
            ord[n++] = (uint8_t)best;
        }
    } else if (nonempty) {
        int best = -1;
        for (uint32_t p = 0; p < P; ++p)
            if (nonempty >> p & 1u)
                if (best < 0 || Q[p] > Q[best]) best = (int)p;
        used |= 1u << best;
        ord[n++] = (uint8_t)best;
    }
    for (uint32_t p = 0; p < P; ++p)
        if (!(used >> p & 1u) && (nonempty >> p & 1u)) {
            used |= 1u << p;
            ord[n++] = (uint8_t)p;
        }
    for (uint32_t p = 0; p < P; ++p)
        if (!(used >> p & 1u)) {
            used |= 1u << p;
            ord[n++] = (uint8_t)p;
        }
    uint32_t start[kMaxPhases];
    uint32_t acc = 0;
    for (uint32_t i = 0; i < P; ++i) {
        order[(size_t)v * kMaxPhases + i] = ord[i];
        start[ord[i]] = acc;
        acc += green[(size_t)v * kMaxPhases + ord[i]];
    }
    for (uint32_t i = P; i < kMaxPhases; ++i) order[(size_t)v * kMaxPhases + i] = (uint8_t)i;
    const uint32_t off = offset[v];
    const unsigned long long magic = ~0ull / cy;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t e = in_edge[i];
        const uint32_t p = ephase[e] & (kMaxPhases - 1);
        EdgeRec& r = rec[e];
        r.cycle = cy;
        r.gbeg = (off + start[p]) % cy;
        r.glen = green[(size_t)v * kMaxPhases + p];
        r.cmagic = magic;
    }
}

// ------------------------------------------------------------------------------------------------
// Batch initialisation: pheromone 1.0 (or Philox-random in [0.5, 1.5)), deposits zero, colony state.
// ------------------------------------------------------------------------------------------------
// Calc_Dist for the whole colony up front: hq[e] = h(head(e)) towards this colony's destination.
__global__ void k_init_batch(uint32_t E, const DevQuery* __restrict__ q, const uint32_t* __restrict__ col,
                             const int32_t* __restrict__ x, const int32_t* __restrict__ y, uint32_t kappa,
                             uint32_t flags, uint64_t* __restrict__ tau, unsigned long long* __restrict__ dep,
                             uint32_t* __restrict__ hq, QueryState* __restrict__ qs, uint32_t* __restrict__ tickets,
                             uint32_t n_tickets) {
    const uint32_t qi = blockIdx.y;
    const DevQuery Q = q[qi];
    uint64_t* T = tau + (size_t)qi * E;
    unsigned long long* D = dep + (size_t)qi * E;
    uint32_t* H = hq + (size_t)qi * E;
    const uint32_t s0 = (uint32_t)Q.seed, s1 = (uint32_t)(Q.seed >> 32);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        uint64_t t0 = 1ull << 32;
        if (flags & GMP_FLAG_RANDOM_TAU) t0 = (1ull << 31) + philox4x32_10(make_uint4(e, 0u, 0u, 1u), s0, s1).x;
        T[e] = t0;
        D[e] = 0;
        const uint32_t v = col[e];
        H[e] = heuristic_ms(x[v], y[v], Q.xd, Q.yd, kappa);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t h = heuristic_ms(x[Q.src], y[Q.src], Q.xd, Q.yd, kappa);
        QueryState S;
        S.best_key = Q.active ? kNoKey : 0ull;
        S.dep_num = (unsigned long long)(h > 0 ? h : 1u) << 32;
        S.steps = 0;
        S.nsucc = 0;
        S.best_len = 0;
        S.best_W = 0;
        S.pad[0] = S.pad[1] = 0;
        qs[qi] = S;
    }
    if (qi == 0 && blockIdx.x == 0)
        for (uint32_t i = threadIdx.x; i < n_tickets; i += blockDim.x) tickets[i] = 0;
}

// ------------------------------------------------------------------------------------------------
// Ant construction. G lanes of a warp serve one ant (sub-warp group); lane l holds the candidates
// l, l+G, ..., l+(K-1)G of the current node's CSR row. Per step: one round of independent 16-byte
// record loads and pheromone loads, scores, a group max, integer weights, a shuffle prefix sum,
// one Philox draw, a ballot to find the chosen road and shuffles to broadcast it.
// Groups take ants from a per-iteration ticket counter, so short walks free lanes for waiting ants.
// ------------------------------------------------------------------------------------------------
template <int G, int K>
__device__ __forceinline__ void walk_ant(const ConstructArgs& a, const DevQuery& q, uint32_t qi, uint32_t k,
                                         uint32_t it, uint32_t* tabu, uint32_t lane, uint32_t gmask, uint32_t gbase) {
    const unsigned long long* __restrict__ tau = reinterpret_cast<const unsigned long long*>(a.tau) +
                                                 (size_t)qi * a.n_edges;
    const uint32_t* __restrict__ hq = a.hq + (size_t)qi * a.n_edges;
    const uint32_t slot = q.ant_base + k;
    uint32_t* route = a.routes + (size_t)slot * a.max_steps;
    const uint32_t s0 = (uint32_t)q.seed, s1 = (uint32_t)(q.seed >> 32);
    uint32_t u = q.src;
    uint32_t beg = __ldg(a.row_ptr + u), end = __ldg(a.row_ptr + u + 1);
    uint32_t t = 0, W = 0, steps = 0, status;
    if (lane == 0) tabu[u >> 5] |= 1u << (u & 31);
    __syncwarp(gmask);
    for (;;) {
        if (u == q.dst) {
            status = kAntSuccess;
            break;
        }
        if (steps == a.max_steps) {
            status = kAntStepCap;
            break;
        }
        const uint32_t deg = end - beg;
        const int nslots = K == 1 ? 1 : (int)((deg + G - 1) / G);  // group-uniform
        // 1. issue every load of this step: records, pheromone and heuristic of this lane's candidates
        uint4 r0[K], r1[K], r2[K];
        unsigned long long te[K];
        uint32_t he[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t idx = lane + (uint32_t)j * G;
            if (j < nslots && idx < deg) {
                const uint4* rp = reinterpret_cast<const uint4*>(a.rec + beg + idx);
                r0[j] = __ldg(rp);
                r1[j] = __ldg(rp + 1);
                r2[j] = __ldg(rp + 2);
                te[j] = __ldg(tau + beg + idx);
                he[j] = __ldg(hq + beg + idx);
            } else {
                r0[j] = r1[j] = r2[j] = make_uint4(0, 0, 0, 0);
                te[j] = 0;
                he[j] = 0;
            }
        }
        // 2. the draw of this step depends on (iteration, ant, step) only: overlaps the loads
        const uint4 o = philox4x32_10(make_uint4(it, k, steps, 0u), s0, s1);
        const unsigned long long rnd = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
        // 3. candidates, waits, scores
        uint32_t cmask = 0, cong = 0;
        uint32_t sb[K], wv[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            sb[j] = wv[j] = 0;
            const uint32_t idx = lane + (uint32_t)j * G;
            if (j < nslots && idx < deg) {
                const uint32_t v = r0[j].x;
                const bool visited = (tabu[v >> 5] >> (v & 31)) & 1u;
                if (!visited) {
                    if (!a.no_prefetch && r0[j].z > r0[j].y) {  // the next step reads one of these rows
                        const char* b0 = reinterpret_cast<const char*>(a.rec + r0[j].y);
                        const char* b1 = reinterpret_cast<const char*>(a.rec + r0[j].z) - 1;
                        for (const char* p = b0; p <= b1; p += 128) prefetch_l1(p);
                        prefetch_l1(b1);
                        prefetch_l1(tau + r0[j].y);
                        prefetch_l1(hq + r0[j].y);
                    }
                    cmask |= 1u << j;
                    if (r2[j].z & 1u) cong |= 1u << j;
                    uint32_t w = 0;
                    const uint32_t cy = r1[j].y;
                    if (v != q.dst && cy != 0) {
                        const unsigned long long mg = (unsigned long long)r2[j].x | ((unsigned long long)r2[j].y << 32);
                        w = signal_wait(a.t_dep + t + r0[j].w, cy, mg, r1[j].z, r1[j].w) + r1[j].x;
                    }
                    wv[j] = w;
                    sb[j] = __float_as_uint(score(te[j], q.alpha, r0[j].w + w + he[j], q.beta));
                }
            }
        }
        if (a.thr_on) {  // congested roads drop out unless every candidate is congested
            const uint32_t any_ok = __ballot_sync(gmask, (cmask & ~cong) != 0u) & gmask;
            const uint32_t any_cg = __ballot_sync(gmask, (cmask & cong) != 0u) & gmask;
            if (any_ok && any_cg) cmask &= ~cong;
        }
        if ((__ballot_sync(gmask, cmask != 0u) & gmask) == 0u) {
            status = kAntDeadEnd;
            break;
        }
        // 4. largest score of the group (non-negative floats order like their bit patterns)
        uint32_t mb = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((cmask >> j & 1u) && sb[j] > mb) mb = sb[j];
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(gmask, mb, off, G));
        uint32_t mmant;
        int mex;
        split_f32(mb, mmant, mex);
        // 5. integer weights and their inclusive prefix in CSR order (index lane + j*G)
        unsigned long long carry = 0, incl[K];
        uint32_t wt[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            wt[j] = 0;
            incl[j] = carry;
            if (j < nslots) {
                wt[j] = (cmask >> j & 1u) ? roulette_weight(sb[j], mmant, mex) : 0u;
                unsigned long long xs = wt[j];
#pragma unroll
                for (int d = 1; d < G; d <<= 1) {
                    const unsigned long long y = __shfl_up_sync(gmask, xs, d, G);
                    if (lane >= (uint32_t)d) xs += y;
                }
                incl[j] = carry + xs;
                if (j + 1 < K) carry += __shfl_sync(gmask, xs, G - 1, G);
                else carry = __shfl_sync(gmask, incl[j], G - 1, G);
            }
        }
        if (K > 1) carry = __shfl_sync(gmask, incl[K - 1], G - 1, G);
        // 6. roulette: first candidate whose running weight exceeds r = floor(rnd * S / 2^64)
        const unsigned long long r = __umul64hi(rnd, carry);
        int js = -1;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (wt[j] != 0u && incl[j] - wt[j] <= r && r < incl[j]) js = j;
        const uint32_t bw = __ballot_sync(gmask, js >= 0) & gmask;
        const int src_lane = (__ffs(bw) - 1) - (int)gbase;
        uint32_t c_idx = 0, c_h = 0, c_vb = 0, c_ve = 0, c_tt = 0, c_w = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (js == j) {
                c_idx = lane + (uint32_t)j * G;
                c_h = r0[j].x;
                c_vb = r0[j].y;
                c_ve = r0[j].z;
                c_tt = r0[j].w;
                c_w = wv[j];
            }
        c_idx = __shfl_sync(gmask, c_idx, src_lane, G);
        c_h = __shfl_sync(gmask, c_h, src_lane, G);
        c_vb = __shfl_sync(gmask, c_vb, src_lane, G);
        c_ve = __shfl_sync(gmask, c_ve, src_lane, G);
        c_tt = __shfl_sync(gmask, c_tt, src_lane, G);
        c_w = __shfl_sync(gmask, c_w, src_lane, G);
        // 7. position update
        const uint32_t e = beg + c_idx;
        t += c_tt + c_w;
        W += c_w;
        u = c_h;
        beg = c_vb;
        end = c_ve;
        if (lane == 0) {
            route[steps] = e;
            tabu[u >> 5] |= 1u << (u & 31);
        }
        ++steps;
        __syncwarp(gmask);
        if (t > kTCap) {
            status = kAntTimeCap;
            break;
        }
    }
    QueryState* S = a.qs + qi;
    if (lane == 0) {
        a.ant_steps[slot] = steps;
        a.ant_wait[slot] = W;
        atomicAdd(&S->steps, (unsigned long long)steps);
        if (status == kAntSuccess) atomicAdd(&S->nsucc, 1ull);
        if (a.ant_log) {
            uint32_t* l = a.ant_log + 4ull * (q.log_base + (uint64_t)it * q.n_ants + k);
            *reinterpret_cast<uint4*>(l) = make_uint4(status, steps, t, W);
        }
    }
    if (status == kAntSuccess) {  // Updt_Pher: deposit dep_num / T on every road of the route
        const unsigned long long delta = S->dep_num / t;
        unsigned long long* D = a.dep + (size_t)qi * a.n_edges;
        for (uint32_t i = lane; i < steps; i += G) atomicAdd(D + route[i], delta);
        if (lane == 0) atomicMin(&S->best_key, ((unsigned long long)t << 32) | ((unsigned long long)it * q.n_ants + k));
    }
    // forget the visited set: whole bitmap when small, else just the nodes of this walk
    if (a.tabu_words <= 2u * (steps + 1u)) {
        for (uint32_t w = lane; w < a.tabu_words; w += G) tabu[w] = 0;
    } else {
        if (lane == 0) atomicAnd(tabu + (q.src >> 5), ~(1u << (q.src & 31)));
        for (uint32_t i = lane; i < steps; i += G) {
            const uint32_t v = __ldg(a.col + route[i]);
            atomicAnd(tabu + (v >> 5), ~(1u << (v & 31)));
        }
    }
    __syncwarp(gmask);
}

template <int G, int K>
__global__ void __launch_bounds__(128) k_construct(ConstructArgs a, uint32_t it) {
    extern __shared__ uint32_t smem[];
    const uint32_t lane = threadIdx.x & (G - 1);
    const uint32_t gib = threadIdx.x / G;
    const uint32_t gbase = (threadIdx.x & 31u) & ~(uint32_t)(G - 1);
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << gbase);
    const uint32_t groups = blockDim.x / G;
    uint32_t* tabu = a.tabu_in_smem ? smem + (size_t)gib * a.tabu_words
                                    : a.tabu_global + ((size_t)blockIdx.x * groups + gib) * a.tabu_words;
    for (uint32_t w = lane; w < a.tabu_words; w += G) tabu[w] = 0;
    __syncwarp(gmask);
    for (;;) {
        uint32_t ticket = 0;
        if (lane == 0) ticket = atomicAdd(a.tickets + it, 1u);
        ticket = __shfl_sync(gmask, ticket, 0, G);
        if (ticket >= a.total_ants) break;
        uint32_t lo = 0, hi = a.n_queries;  // query with ant_prefix[q] <= ticket < ant_prefix[q + 1]
        while (hi - lo > 1u) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(a.ant_prefix + mid) <= ticket) lo = mid;
            else hi = mid;
        }
        const DevQuery q = a.queries[lo];
        if (!q.active || it >= q.n_iter) continue;
        walk_ant<G, K>(a, q, lo, ticket - q.ant_base, it, tabu, lane, gmask, gbase);
    }
}

// ------------------------------------------------------------------------------------------------
// Evap_Pher + Updt_Pher: tau <- tau - floor(tau * rho_fix / 2^32) + D ; D <- 0.
// ------------------------------------------------------------------------------------------------
__global__ void k_evaporate(uint32_t E, const DevQuery* __restrict__ q, uint64_t* __restrict__ tau,
                            unsigned long long* __restrict__ dep, uint32_t it) {
    const uint32_t qi = blockIdx.y;
    const uint32_t active = q[qi].active, n_iter = q[qi].n_iter;
    if (!active || it >= n_iter) return;
    const uint64_t rf = q[qi].rho_fix;
    uint64_t* T = tau + (size_t)qi * E;
    unsigned long long* D = dep + (size_t)qi * E;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const uint64_t t = T[e];
        const uint64_t lo = t * rf, hi = __umul64hi(t, rf);
        T[e] = t - ((hi << 32) | (lo >> 32)) + D[e];
        D[e] = 0;
    }
}

// Best-route tracking: when the colony's best key came from this iteration, keep that ant's route.
__global__ void k_best_copy(const DevQuery* __restrict__ q, QueryState* __restrict__ qs,
                            const uint32_t* __restrict__ routes, const uint32_t* __restrict__ ant_steps,
                            const uint32_t* __restrict__ ant_wait, uint32_t* __restrict__ best_route,
                            uint32_t max_steps, uint32_t it) {
    const uint32_t qi = blockIdx.x;
    const DevQuery Q = q[qi];
    if (!Q.active || it >= Q.n_iter) return;
    const unsigned long long key = qs[qi].best_key;
    if (key == kNoKey) return;
    const uint32_t low = (uint32_t)key;
    if (low / Q.n_ants != it) return;
    const uint32_t slot = Q.ant_base + low % Q.n_ants;
    const uint32_t len = ant_steps[slot];
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
        best_route[(size_t)qi * max_steps + i] = routes[(size_t)slot * max_steps + i];
    if (threadIdx.x == 0) {
        qs[qi].best_len = len;
        qs[qi].best_W = ant_wait[slot];
    }
}

__global__ void k_finalize(const DevQuery* __restrict__ q, const QueryState* __restrict__ qs,
                           const uint32_t* __restrict__ best_route, const uint32_t* __restrict__ col,
                           uint32_t max_steps, DevResult* __restrict__ res, uint32_t* __restrict__ route_out) {
    const uint32_t qi = blockIdx.x;
    const DevQuery Q = q[qi];
    const QueryState S = qs[qi];
    const bool found = S.best_key != kNoKey;
    if (threadIdx.x == 0) {
        DevResult r;
        r.ant_steps = S.steps;
        r.n_success = S.nsucc;
        r.status = found ? GMP_OK : GMP_ERR_NO_ROUTE;
        r.travel_ms = found ? (S.best_key >> 32) : 0;
        r.wait_ms = found ? S.best_W : 0;
        r.route_len = found ? S.best_len + 1 : 0;
        const uint32_t low = (uint32_t)S.best_key;
        r.best_iter = (found && Q.active) ? low / Q.n_ants : 0;
        r.best_ant = (found && Q.active) ? low % Q.n_ants : 0;
        res[qi] = r;
    }
    if (!found) return;
    uint32_t* out = route_out + (size_t)qi * (max_steps + 1);
    if (threadIdx.x == 0) out[0] = Q.src;
    for (uint32_t i = threadIdx.x; i < S.best_len; i += blockDim.x)
        out[i + 1] = col[best_route[(size_t)qi * max_steps + i]];
}

// ------------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------------
static inline unsigned blocks_for(uint64_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_edge_static(cudaStream_t s, uint32_t E, const uint32_t* len, const uint16_t* speed,
                               const uint8_t* lanes, uint32_t* ff, uint32_t* cap) {
    if (E == 0) return cudaSuccess;
    k_edge_static<<<blocks_for(E, 256), 256, 0, s>>>(E, len, speed, lanes, ff, cap);
    return cudaGetLastError();
}

cudaError_t launch_edge_dynamic(cudaStream_t s, uint32_t E, const uint32_t* row_ptr, const uint32_t* col,
                                const uint32_t* ff, const uint32_t* cap, const uint8_t* lanes, const uint32_t* veh,
                                const uint8_t* nph, uint32_t h_sat, uint32_t thr, EdgeRec* rec) {
    if (E == 0) return cudaSuccess;
    k_edge_dynamic<<<blocks_for(E, 256), 256, 0, s>>>(E, row_ptr, col, ff, cap, lanes, veh, nph, h_sat, thr, rec);
    return cudaGetLastError();
}

cudaError_t launch_queue_preempt(cudaStream_t s, uint32_t N, const uint32_t* in_ptr, const uint32_t* in_edge,
                                 const uint8_t* nph, const uint32_t* cycle, const uint32_t* offset,
                                 const uint32_t* green, const uint8_t* ephase, const uint32_t* veh,
                                 const uint32_t* cap, const uint32_t* red, uint8_t* order, EdgeRec* rec) {
    if (N == 0) return cudaSuccess;
    k_queue_preempt<<<blocks_for(N, 128), 128, 0, s>>>(N, in_ptr, in_edge, nph, cycle, offset, green, ephase, veh,
                                                        cap, red, order, rec);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(cudaStream_t s, uint32_t Q, uint32_t E, const DevQuery* q, const uint32_t* col,
                              const int32_t* x, const int32_t* y, uint32_t kappa, uint32_t flags, uint64_t* tau,
                              unsigned long long* dep, uint32_t* hq, QueryState* qs, uint32_t* tickets,
                              uint32_t n_tickets) {
    dim3 grid(blocks_for(E ? E : 1, 1024), Q);
    k_init_batch<<<grid, 256, 0, s>>>(E, q, col, x, y, kappa, flags, tau, dep, hq, qs, tickets, n_tickets);
    return cudaGetLastError();
}

cudaError_t launch_evaporate(cudaStream_t s, uint32_t Q, uint32_t E, const DevQuery* q, uint64_t* tau,
                             unsigned long long* dep, uint32_t it) {
    if (E == 0) return cudaSuccess;
    dim3 grid(blocks_for(E, 1024), Q);
    k_evaporate<<<grid, 256, 0, s>>>(E, q, tau, dep, it);
    return cudaGetLastError();
}

cudaError_t launch_best_copy(cudaStream_t s, uint32_t Q, const DevQuery* q, QueryState* qs, const uint32_t* routes,
                             const uint32_t* ant_steps, const uint32_t* ant_wait, uint32_t* best_route,
                             uint32_t max_steps, uint32_t it) {
    k_best_copy<<<Q, 128, 0, s>>>(q, qs, routes, ant_steps, ant_wait, best_route, max_steps, it);
    return cudaGetLastError();
}

cudaError_t launch_finalize(cudaStream_t s, uint32_t Q, const DevQuery* q, const QueryState* qs,
                            const uint32_t* best_route, const uint32_t* col, uint32_t max_steps, DevResult* res,
                            uint32_t* route_out) {
    k_finalize<<<Q, 128, 0, s>>>(q, qs, best_route, col, max_steps, res, route_out);
    return cudaGetLastError();
}

template <int G, int K>
static cudaError_t config_for(int device, uint32_t n_nodes, uint32_t total_ants, KernelConfig* out) {
    const int block = 128;
    const int groups = block / G;
    const uint32_t words = (n_nodes + 31u) / 32u;
    const size_t smem = (size_t)groups * words * 4u;
    const bool in_smem = smem <= 64u * 1024u;
    const size_t dyn = in_smem ? smem : 0;
    cudaError_t err;
    if (dyn > 48u * 1024u) {
        err = cudaFuncSetAttribute(k_construct<G, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (err != cudaSuccess) return err;
    }
    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct<G, K>, block, dyn);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    const uint64_t need = ((uint64_t)total_ants + groups - 1) / groups;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    out->lanes = G;
    out->slots = K;
    out->block = block;
    out->grid = (int)grid;
    out->smem = dyn;
    out->tabu_in_smem = in_smem;
    return cudaSuccess;
}

// Candidate slots per lane: the fewest of {1, 2, 4} that cover the largest out-degree.
static int slots_for(int lanes, uint32_t max_degree) {
    for (int k : {1, 2, 4})
        if ((uint32_t)(lanes * k) >= max_degree) return k;
    return 0;
}

int construct_max_degree(int lanes) { return lanes * 4; }

cudaError_t construct_config(int device, int lanes, uint32_t n_nodes, uint32_t max_degree, uint32_t total_ants,
                             KernelConfig* out) {
    const int k = slots_for(lanes, max_degree);
#define GMP_CFG(G_, K_) \
    if (lanes == G_ && k == K_) return config_for<G_, K_>(device, n_nodes, total_ants, out);
    GMP_CFG(4, 1) GMP_CFG(4, 2) GMP_CFG(4, 4) GMP_CFG(8, 1) GMP_CFG(8, 2) GMP_CFG(8, 4)
    GMP_CFG(16, 1) GMP_CFG(16, 2) GMP_CFG(16, 4) GMP_CFG(32, 1) GMP_CFG(32, 2) GMP_CFG(32, 4)
#undef GMP_CFG
    return cudaErrorInvalidValue;
}

cudaError_t launch_construct(cudaStream_t s, const KernelConfig& kc, const ConstructArgs& a, uint32_t it) {
#define GMP_LAUNCH(G_, K_)                                                    \
    if (kc.lanes == G_ && kc.slots == K_) {                                   \
        k_construct<G_, K_><<<kc.grid, kc.block, kc.smem, s>>>(a, it);        \
        return cudaGetLastError();                                            \
    }
    GMP_LAUNCH(4, 1) GMP_LAUNCH(4, 2) GMP_LAUNCH(4, 4) GMP_LAUNCH(8, 1) GMP_LAUNCH(8, 2) GMP_LAUNCH(8, 4)
    GMP_LAUNCH(16, 1) GMP_LAUNCH(16, 2) GMP_LAUNCH(16, 4) GMP_LAUNCH(32, 1) GMP_LAUNCH(32, 2) GMP_LAUNCH(32, 4)
#undef GMP_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace gmp

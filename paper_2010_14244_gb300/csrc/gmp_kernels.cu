// sm_103a kernels of the MACO-P route colony (Jindal & Bedi, GMACO-P, Sec. 4.2, Algorithm 2).
//
//   k_edge_static     road free-flow time and jam capacity, per approach slot           (graph load)
//   k_queue_small     per-intersection phase order by the preemptive rule, and the road records of
//   k_queue_general   its approaches (congested time, queue delay, green window)     (Calc_Dens, Comp_Thres)
//   k_tick_node       serving tick: discharge of every approach and red-time update  (Fig. 3 signal block)
//   k_init_batch      initial pheromone, per-colony state                          (Algorithm 2)
//   k_construct<G,K>  ant walks: Adj_Neigh, next-node roulette, Eval_Rout, position update, deposits
//   k_construct_tail  the walks a construction launch handed off after handoff_moves moves, finished
//                     one per warp by the pipelined walk (walk_ant_spec)
//   k_iter_end        Evap_Pher fused with the deposits of Updt_Pher, best-route tracking and the
//                     per-iteration queue/preemption update, in one launch
//   k_finalize        best route as node ids + counters
#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp_device.cuh"
#include "gmp_internal.h"
#include "gmp_walk.cuh"

namespace gmp {

// ------------------------------------------------------------------------------------------------
// Road attributes, per approach slot (slot i holds road in_edge[i])
// ------------------------------------------------------------------------------------------------
__global__ void k_edge_static(uint32_t E, const uint32_t* __restrict__ in_edge, const uint32_t* __restrict__ len,
                              const uint16_t* __restrict__ speed, const uint8_t* __restrict__ lanes_by_road,
                              uint32_t* __restrict__ ff, uint32_t* __restrict__ cap, uint8_t* __restrict__ lanes) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E) return;
    const uint32_t e = in_edge[i];
    const uint64_t L = len[e], v = speed[e], ln = lanes_by_road[e];
    uint64_t f = (L * 360u + v / 2u) / v;  // length / speed in ms, rounded half up
    f = f < 1u ? 1u : (f > kTimeClamp ? kTimeClamp : f);
    ff[i] = (uint32_t)f;
    const uint64_t c = ln * L / 75u;  // one vehicle per 7.5 m of lane
    cap[i] = c < 1u ? 1u : (uint32_t)c;
    lanes[i] = (uint8_t)ln;
}

template <class T>
__global__ void k_gather(uint32_t n, const uint32_t* __restrict__ idx, const T* __restrict__ src, T* __restrict__ dst) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// ------------------------------------------------------------------------------------------------
// Preemptive phase order, one thread per intersection (queue_node_small / queue_node in gmp_walk.cuh):
// the small kernel covers the intersections with at most two phases, the general one the others.
// ------------------------------------------------------------------------------------------------
template <bool FULL, bool TICK>
__global__ void __launch_bounds__(128) k_queue_small(QueueTables t) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < t.n_nodes) queue_node_small<FULL, TICK>(v, t);
}

template <bool FULL, bool TICK>
__global__ void __launch_bounds__(128) k_queue_general(QueueTables t) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < t.n_nodes && t.nph[v] > 2u) queue_node<FULL, TICK>(v, t);
}

// ------------------------------------------------------------------------------------------------
// Serving tick: the queue/preemption update with dt > 0 (Fig. 3 signal block, Calc_Dens and Comp_Thres
// of Sec. 4.2 applied to moving vehicles). The node pass below, then a queue pass that first moves the
// discharged vehicles on (approach_vehicles in gmp_walk.cuh) and rebuilds the phase orders and records.
// ------------------------------------------------------------------------------------------------
// Saturation discharge of one lane count over the tick, lanes * (t + dt) / h_sat - lanes * t / h_sat
// vehicles (the whole clock counts), per lane count 0..255, capped at 2^32 - 1.
struct TickCap {
    uint32_t cap[256];
};

// Node pass (one thread per node, over its approaches): the phase green at t_now under the current
// order (every approach is served at an unsignalised node), the discharge of every served approach, the
// node's total discharge, and its red-time update for phases below red_planes: 0 for the green phase, for
// phases without a queue and at or above the node's phase count, + dt saturating otherwise (queues
// before the discharge). The node's own words (its phase planes below red_planes exist for every node)
// are loaded together, then its approaches four at a time.
__global__ void __launch_bounds__(128) k_tick_node(QueueTables t, uint64_t t_now, uint32_t dt, uint32_t red_planes,
                                                   TickCap tc, uint32_t* __restrict__ leave,
                                                   unsigned long long* __restrict__ K) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.n_nodes) return;
    const uint32_t N = t.n_nodes;
    const uint32_t P = t.nph[v], ib = t.in_ptr[v], ie = t.in_ptr[v + 1];
    const uint32_t cy = t.cycle[v], off = t.offset[v];
    const uint2 o = *reinterpret_cast<const uint2*>(t.order + (size_t)v * kMaxPhases);
    uint32_t g[kMaxPhases], rd[kMaxPhases];
#pragma unroll
    for (uint32_t p = 0; p < kMaxPhases; ++p) {
        g[p] = p < red_planes ? t.green[(size_t)p * N + v] : 0u;
        rd[p] = p < red_planes ? t.red[(size_t)p * N + v] : 0u;
    }
    uint32_t gph = 0xFFFFFFFFu;
    if (P) {
        const uint32_t c = (uint32_t)((t_now % cy + cy - off % cy) % cy);  // position in the cycle
        uint32_t start = 0;
#pragma unroll
        for (uint32_t i = 0; i < kMaxPhases; ++i) {
            if (i < P && gph == 0xFFFFFFFFu) {
                const uint32_t p = ((i < 4u ? o.x : o.y) >> (8u * (i & 3u))) & 0xFFu;
                uint32_t gp = 0;
#pragma unroll
                for (uint32_t q = 0; q < kMaxPhases; ++q) gp = q == p ? g[q] : gp;
                if (c >= start && c < start + gp) gph = p;
                start += gp;
            }
        }
    }
    uint32_t nonempty = 0;  // phases with vehicles on some approach
    unsigned long long k = 0;
    for (uint32_t i0 = ib; i0 < ie; i0 += 4) {
        const uint32_t m = ie - i0 < 4u ? ie - i0 : 4u;
        uint32_t n[4], ph[4], ln[4];
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const bool ok = j < m;
            n[j] = ok ? t.veh[i0 + j] : 0u;
            ph[j] = ok ? t.ephase[i0 + j] : 0u;
            ln[j] = ok ? t.lanes[i0 + j] : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            if (j < m) {
                nonempty |= (n[j] > 0u ? 1u : 0u) << (ph[j] & (kMaxPhases - 1));
                uint32_t out = 0;
                if (P == 0 || ph[j] == gph) {
                    const uint32_t cap = tc.cap[ln[j]];
                    out = n[j] < cap ? n[j] : cap;
                }
                leave[i0 + j] = out;
                k += out;
            }
        }
    }
    K[v] = k;
#pragma unroll
    for (uint32_t p = 0; p < kMaxPhases; ++p) {
        if (p < red_planes) {
            const bool keep = P != 0 && p < P && p != gph && (nonempty >> p & 1u);
            t.red[(size_t)p * N + v] = keep ? (rd[p] > 0xFFFFFFFFu - dt ? 0xFFFFFFFFu : rd[p] + dt) : 0u;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Exact Calc_Dist (GMP_FLAG_EXACT_H): per colony, h(v) = the least sum of congested travel times over
// the roads of a path from v to the colony's destination, saturating at 2^28 (also for nodes that
// cannot reach it). One block per colony relaxes from the destination over the reversed roads with
// atomicMin on the bounds, in near-far order (Davidson, Baxter, Garland & Owens, IPDPS 2014): a level
// relaxes the near frontier; a node it lowers below the threshold T joins the next near frontier (once
// per level: stamped with the level), one lowered to T or above joins the far pile (once per epoch:
// stamped with the epoch). When the near frontier runs dry, T grows to max(T + delta, least far bound
// + delta) and the far nodes below it become the next frontier; the rest stay far. The saturating sums
// are monotone, so the fixpoint is the clamped exact distance in any relaxation order: delta and the
// order only change the amount of work. Each epoch settles at least one node; a colony that runs past
// 4N + 4096 levels (far beyond anything observed) sets err[0] and stops.
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kExactHBlock = 512;

__global__ void __launch_bounds__(kExactHBlock, 4)
k_exact_h(uint32_t N, const DevQuery* __restrict__ q, const uint32_t* __restrict__ in_ptr,
          const uint32_t* __restrict__ in_edge, const uint32_t* __restrict__ in_tail, const EdgeRec* __restrict__ rec,
          uint32_t delta, uint32_t level_limit, uint32_t* hdist, uint32_t* queue, uint32_t* stamps, uint32_t* err) {
    const uint32_t qi = blockIdx.x;
    const uint32_t dst = q[qi].dst;
    uint32_t* dist = hdist + (size_t)qi * N;
    uint32_t* nstamp = stamps + (size_t)qi * 2u * N;  // near: level + 1 of the frontier a node last joined
    uint32_t* fstamp = nstamp + N;                    // far: epoch + 1 of the pile a node last joined
    uint32_t* qa = queue + (size_t)qi * 4u * N;       // near frontier of this level
    uint32_t* qb = qa + N;                            // near frontier of the next level
    uint32_t* fa = qb + N;                            // far pile of this epoch
    uint32_t* fb = fa + N;                            // far pile of the next epoch
    __shared__ uint32_t ncnt[2], fcnt[2], fmin;
    for (uint32_t v = threadIdx.x; v < N; v += blockDim.x) {
        dist[v] = kHClamp;
        nstamp[v] = 0;
        fstamp[v] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        dist[dst] = 0;
        qa[0] = dst;  // frontier of level 0 (stamp 0)
        ncnt[0] = 1;
        ncnt[1] = 0;
        fcnt[0] = 0;
        fcnt[1] = 0;
        fmin = 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t guard = level_limit ? level_limit : (N > (1u << 29) ? 0xFFFFFFFFu : 4u * N + 4096u);
    uint32_t T = delta, epoch = 0, fsel = 0;
    for (uint32_t level = 0;; ++level) {
        if (level > guard) {
            if (threadIdx.x == 0) atomicExch(err, 1u);
            return;
        }
        const uint32_t n_cur = ncnt[level & 1u];
        const uint32_t nf = fcnt[fsel];
        if (n_cur == 0 && nf == 0) break;
        __syncthreads();  // every thread has read this level's counts
        if (threadIdx.x == 0) ncnt[level & 1u] = 0;  // the counter of the near frontier of level + 2
        uint32_t* const next_cnt = ncnt + ((level + 1u) & 1u);
        const uint32_t mark = level + 1u;
        if (n_cur == 0) {  // the near frontier ran dry: a new epoch splits the far pile
            uint32_t* const far_cur = fsel ? fb : fa;
            uint32_t* const far_nxt = fsel ? fa : fb;
            for (uint32_t i = threadIdx.x; i < nf; i += blockDim.x) atomicMin(&fmin, __ldcg(dist + far_cur[i]));
            __syncthreads();
            const uint32_t lo = fmin;  // below 2^28: far nodes were lowered below the clamp
            T = max(T + delta, lo + delta);
            ++epoch;
            const uint32_t fmark = epoch + 1u;
            for (uint32_t i = threadIdx.x; i < nf; i += blockDim.x) {
                const uint32_t v = far_cur[i];
                if (__ldcg(dist + v) < T) {
                    if (atomicExch(nstamp + v, mark) != mark) qb[atomicAdd(next_cnt, 1u)] = v;
                } else if (atomicExch(fstamp + v, fmark) != fmark) {
                    far_nxt[atomicAdd(&fcnt[fsel ^ 1u], 1u)] = v;
                }
            }
            __syncthreads();  // the split is complete; every thread has read fmin and fcnt[fsel]
            if (threadIdx.x == 0) {
                fcnt[fsel] = 0;
                fmin = 0xFFFFFFFFu;
            }
            fsel ^= 1u;
        } else {
            uint32_t* const far_cur = fsel ? fb : fa;
            const uint32_t fmark = epoch + 1u;
            for (uint32_t i = threadIdx.x; i < n_cur; i += blockDim.x) {
                const uint32_t u = qa[i];
                const uint32_t du = __ldcg(dist + u);  // bounds change by atomics (in L2): skip L1
                const uint32_t k1 = in_ptr[u + 1];
                for (uint32_t k0 = in_ptr[u]; k0 < k1; k0 += 4) {
                    // up to four in-roads: every load first, then the atomics of the relaxations that
                    // improve on the bound read (most do not; a stale read only costs an atomic)
                    uint32_t vv[4], nd[4], cur[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool ok = k0 + j < k1;
                        vv[j] = ok ? in_tail[k0 + j] : 0u;
                        nd[j] = ok ? min(du + rec[in_edge[k0 + j]].tt, kHClamp) : kHClamp;
                        cur[j] = ok ? __ldcg(dist + vv[j]) : 0u;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (!(nd[j] < cur[j] && nd[j] < atomicMin(dist + vv[j], nd[j]))) continue;
                        if (nd[j] < T) {
                            if (atomicExch(nstamp + vv[j], mark) != mark) qb[atomicAdd(next_cnt, 1u)] = vv[j];
                        } else if (atomicExch(fstamp + vv[j], fmark) != fmark) {
                            far_cur[atomicAdd(&fcnt[fsel], 1u)] = vv[j];
                        }
                    }
                }
            }
        }
        uint32_t* const t = qa;
        qa = qb;
        qb = t;
        __syncthreads();  // the next near frontier (and far pile) is complete
    }
}

// ------------------------------------------------------------------------------------------------
// Batch initialisation: pheromone 1.0 (or Philox-random in [0.5, 1.5)), colony state, and with zero_dep the
// deposit accumulators (an iterative job leaves them zero: every iteration end clears the deposits it
// applies, and a road only receives deposits in an iteration whose end processes it).
// ------------------------------------------------------------------------------------------------
// Calc_Dist for the whole colony up front: th[e].y = h(head(e)) towards this colony's destination,
// next to th[e].x, the pheromone as binary32 bits (one 8-byte load per candidate). h is the
// straight-line bound, or with EXACT (GMP_FLAG_EXACT_H) the colony's row of hdist (N per colony). EXACT
// and REP (GMP_FLAG_REPULSIVE: the pheromone word is a reciprocal) are template parameters so that the
// default instantiation keeps its small register footprint: this kernel writes every road of every
// colony and needs the occupancy.
constexpr uint32_t kInitCols = 8;  // colonies per thread: a road's head and coordinates are read once for them

// One thread per road and group of kInitCols colonies (blockIdx.y): the head and its coordinates are
// loaded once, then each colony's bound and pair are computed and written (each colony's pairs are
// contiguous, so a warp's writes for one colony are one run).
template <bool EXACT, bool REP>
__global__ void __launch_bounds__(256, EXACT ? 6 : 8)
k_init_batch(uint32_t Qn, uint32_t E, const DevQuery* __restrict__ q, const uint32_t* __restrict__ col,
             const int32_t* __restrict__ x, const int32_t* __restrict__ y, uint32_t kappa,
             uint32_t flags, uint64_t* __restrict__ tau, uint2* __restrict__ th,
             unsigned long long* __restrict__ dep, QueryState* __restrict__ qs,
             uint32_t* __restrict__ tickets, uint32_t n_tickets, uint32_t sparse,
             uint32_t* __restrict__ tflag, uint32_t tflag_words,
             const uint32_t* __restrict__ hdist, uint32_t N, uint32_t zero_dep) {
    const uint32_t q0 = blockIdx.y * kInitCols, q1 = min(Qn, q0 + kInitCols);
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E) {
        const uint32_t v = col[e];
        const int32_t xv = EXACT ? 0 : x[v], yv = EXACT ? 0 : y[v];
        for (uint32_t qi = q0; qi < q1; ++qi) {
            const uint32_t h = EXACT ? hdist[(size_t)qi * N + v] : heuristic_ms(xv, yv, q[qi].xd, q[qi].yd, kappa);
            const size_t o = (size_t)qi * E + e;
            if (zero_dep) dep[o] = 0;
            if (sparse) {  // no road has a deposit yet: every road holds the baseline
                th[o] = make_uint2(0u, h);
                continue;
            }
            uint64_t t0 = 1ull << 32;
            if (flags & GMP_FLAG_RANDOM_TAU) {
                const uint64_t seed = q[qi].seed;
                t0 = (1ull << 31) + philox4x32_10(make_uint4(e, 0u, 0u, 1u), (uint32_t)seed, (uint32_t)(seed >> 32)).x;
            }
            tau[o] = t0;
            th[o] = make_uint2(tau_word(t0, REP ? GMP_FLAG_REPULSIVE : 0u), h);
        }
    }
    if (sparse)
        for (uint32_t qi = q0; qi < q1; ++qi)
            for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < tflag_words; w += gridDim.x * blockDim.x)
                tflag[(size_t)qi * tflag_words + w] = 0;
    if (blockIdx.x == 0 && threadIdx.x < q1 - q0) {
        const uint32_t qi = q0 + threadIdx.x;
        const DevQuery Q = q[qi];
        const uint32_t h = EXACT ? hdist[(size_t)qi * N + Q.src] : heuristic_ms(x[Q.src], y[Q.src], Q.xd, Q.yd, kappa);
        QueryState S;
        S.best_key = Q.active ? kNoKey : 0ull;
        S.dep_num = (flags & GMP_FLAG_UNIT_DEPOSIT) ? 0ull : (unsigned long long)(h > 0 ? h : 1u) << 32;
        S.steps = 0;
        S.nsucc = 0;
        S.best_len = 0;
        S.best_W = 0;
        S.h_src = h;
        S.pad = 0;
        S.base_tau = 1ull << 32;
        S.base_tf = tau_word(1ull << 32, REP ? GMP_FLAG_REPULSIVE : 0u);
        S.n_touched = 0;
        qs[qi] = S;
    }
    if (blockIdx.y == 0 && blockIdx.x == 0)
        for (uint32_t i = threadIdx.x; i < n_tickets; i += blockDim.x) tickets[i] = 0;
}

template <int G, int K, bool SMEM>
__global__ void __launch_bounds__(128) k_construct(ConstructArgs a, uint32_t it) {
    extern __shared__ uint32_t smem[];
    const uint32_t lane = threadIdx.x & (G - 1);
    const uint32_t gib = threadIdx.x / G;
    const uint32_t gbase = (threadIdx.x & 31u) & ~(uint32_t)(G - 1);
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << gbase);
    const uint32_t groups = blockDim.x / G;
    uint32_t* tabu = SMEM ? smem + (size_t)gib * a.tabu_words
                          : a.tabu_global + ((size_t)blockIdx.x * groups + gib) * a.tabu_words;
    // shared bitmaps start uncleared; global ones are cleared once per job and every walk clears its
    // own bits when it ends
    if (SMEM)
        for (uint32_t w = lane; w < a.tabu_words; w += G) tabu[w] = 0;
    __syncwarp(gmask);
    for (;;) {
        uint32_t ticket = 0;
        if (lane == 0) ticket = atomicAdd(a.tickets + it, 1u);
        ticket = __shfl_sync(gmask, ticket, 0, G);
        if (ticket >= a.total_ants) break;
        const uint32_t tg = a.ticket_base + ticket;  // the ant's index in the whole job
        uint32_t lo = 0, hi = a.n_queries;  // query with ant_prefix[q] <= tg < ant_prefix[q + 1]
        while (hi - lo > 1u) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(a.ant_prefix + mid) <= tg) lo = mid;
            else hi = mid;
        }
        const DevQuery q = a.queries[lo];
        if (!q.active || it >= q.n_iter) continue;
        walk_ant<G, K, SMEM, SMEM>(a, q, lo, tg - q.ant_base, it, tabu, lane, gmask, gbase);  // hand-off: shared bitmaps
    }
}

// Tail of an iteration's construction (handoff_moves != 0): the walks the construction launch suspended,
// finished one per warp by the pipelined walk. Warps take walks from a counter; each copies its walk's
// visited set into its slice of shared memory first.
__global__ void __launch_bounds__(128) k_construct_tail(ConstructArgs a, uint32_t it) {
    extern __shared__ uint32_t smem[];
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t* tabu = smem + (size_t)(threadIdx.x >> 5) * a.tabu_words;
    const uint32_t n = a.tail_count[it];  // final: the construction launch before this one wrote it
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(a.tail_claim + it, 1u);
        i = __shfl_sync(FULL, i, 0);
        if (i >= n) break;
        const uint32_t slot = a.tail_list[a.ticket_base + i];
        const WalkState ws = a.tail_state[slot];
        const uint32_t* in = a.tail_tabu + (size_t)slot * a.tabu_words;
        for (uint32_t w = lane; w < a.tabu_words; w += 32u) tabu[w] = in[w];
        __syncwarp();
        const DevQuery q = a.queries[ws.qi];
        walk_ant_spec(a, q, ws.qi, ws.k, it, tabu, lane, ws);
    }
}

// ------------------------------------------------------------------------------------------------
// Ant construction, G lanes per ant, all ants of a warp in lockstep: every loop iteration each of the
// 32/G groups advances its ant by one step through the same code, so one warp instruction serves all
// of them (a warp whose groups wander apart would issue each group's instructions separately). Row
// loads stay coalesced within a group. Shuffles run on the full warp with width G. A group whose ant
// ended finalises it (deposits and bitmap reset spread over its G lanes) and takes a new ant; new ants
// come from one warp-aggregated atomic per round. The loads of an ant's next row are issued as soon as
// it moves, so their latency overlaps the end of the step and the loop's bookkeeping.
// ------------------------------------------------------------------------------------------------
template <int G, int K, bool SMEM, bool FRAC>
__global__ void __launch_bounds__(128) k_construct_gl(ConstructArgs a, uint32_t it) {
    extern __shared__ uint32_t smem[];
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    constexpr int NC = G * K;
    const uint32_t lane = threadIdx.x & (G - 1);       // lane within the group
    const uint32_t wl = threadIdx.x & 31u;             // lane within the warp
    const uint32_t gib = threadIdx.x / G;
    const uint32_t groups = blockDim.x / G;
    const bool leader = lane == 0;
    uint32_t* const tabu = SMEM ? smem + (size_t)gib * a.tabu_words
                                : a.tabu_global + ((size_t)blockIdx.x * groups + gib) * a.tabu_words;
    // shared bitmaps start uncleared; global ones are cleared once per job and every walk clears its
    // own bits when it ends
    if (SMEM)
        for (uint32_t w = lane; w < a.tabu_words; w += G) tabu[w] = 0;
    __syncwarp();
    const uint32_t lt_mask = (1u << wl) - 1u;
    bool active = false, exhausted = false;
    uint32_t qi = 0, k = 0, slot = 0, src = 0, dst = 0, n_ants = 1, alpha = 1, beta = 2, s0 = 0, s1 = 0;
    bool frac = false;  // non-integer exponents (FRAC instantiations only): alpha and beta are binary32 bits
    uint64_t log_base = 0;
    uint32_t u = 0, beg = 0, end = 0, t = 0, W = 0, steps = 0, status = 0;
    uint32_t len = 0, pops = 0, hu = 0;  // roads in the route, steps back so far, remaining bound at u
    // Philox draws of the next G steps, one per lane: lane l holds the draw of step rb_base + l
    uint32_t rb_base = 0, rb_x = 0, rb_y = 0;
    bool rb_valid = false;
    const uint2* th = a.th;
    float base_tf = 0.0f;  // sparse layout: the colony's baseline pheromone of this iteration
    uint32_t* route = a.routes;
    uint32_t* rwait = a.rwait;
    bool want = true;  // warp-uniform: some group may need a ticket (at the start, after an ant ended)
    // the next step's candidate loads, issued as soon as the ant moves (software pipelining)
    uint4 p0[K], p1[K];
    uint2 pth[K];
    bool pre = false;
    for (;;) {
        // 1. groups without an ant take the next tickets (one atomic for the whole warp)
        const bool need = !active && !exhausted;
        const uint32_t nmask = want ? __ballot_sync(FULL, need && leader) : 0u;
        if (nmask) {
            const int first = __ffs(nmask) - 1;
            uint32_t base = 0;
            if ((int)wl == first) base = atomicAdd(a.tickets + it, (uint32_t)__popc(nmask));
            base = __shfl_sync(FULL, base, first);
            uint32_t tk = base + (uint32_t)__popc(nmask & lt_mask);
            tk = __shfl_sync(FULL, tk, 0, G);  // the group's leader holds the group's ticket
            if (need) {
                if (tk >= a.total_ants) {
                    exhausted = true;
                } else {
                    const uint32_t tg = a.ticket_base + tk;  // the ant's index in the whole job
                    uint32_t lo = 0, hi = a.n_queries;  // query with ant_prefix[q] <= tg < ant_prefix[q + 1]
                    while (hi - lo > 1u) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (__ldg(a.ant_prefix + mid) <= tg) lo = mid;
                        else hi = mid;
                    }
                    const DevQuery q = a.queries[lo];
                    if (q.active && it < q.n_iter) {
                        active = true;
                        qi = lo;
                        k = tg - q.ant_base;
                        slot = tg;
                        src = q.src;
                        dst = q.dst;
                        n_ants = q.n_ants;
                        alpha = q.alpha;
                        beta = q.beta;
                        frac = FRAC && (q.active & kQueryFracExp) != 0u;
                        s0 = (uint32_t)q.seed;
                        s1 = (uint32_t)(q.seed >> 32);
                        log_base = q.log_base;
                        th = a.th + (size_t)qi * a.n_edges;
                        base_tf = a.sparse ? __uint_as_float(a.qs[qi].base_tf) : 0.0f;
                        route = a.routes + (size_t)slot * a.max_steps;
                        rwait = a.rwait + (size_t)slot * a.max_steps;
                        u = src;
                        beg = __ldg(a.row_ptr + u);
                        end = __ldg(a.row_ptr + u + 1);
                        hu = a.qs[qi].h_src;
                        t = W = steps = len = pops = 0;
                        rb_valid = false;
                        pre = false;
                        if (leader) atomicOr(tabu + (u >> 5), 1u << (u & 31));
                    }
                }
            }
            __syncwarp();
        }
        if (want) want = __any_sync(FULL, !active && !exhausted);  // tickets of colonies without work
        if (!__any_sync(FULL, active)) {
            if (want) continue;
            break;  // no ant and no tickets left
        }
        // 2. one step of every active ant
        bool done = false;
        if (active && u == dst) {
            done = true;
            status = kAntSuccess;
        } else if (active && steps == a.max_steps) {
            done = true;
            status = kAntStepCap;
        }
        const bool stepping = active && !done;
        const uint32_t deg = stepping ? end - beg : 0u;
        const int nslots = K == 1 ? 1 : (int)__reduce_max_sync(FULL, (deg + G - 1) / G);  // warp-uniform
        {  // runs for every warp with an active ant (a warp whose ants all just ended masks everything)
            uint4 r0[K], r1[K];
            float tf[K];
            uint32_t he[K];
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {  // slots past a row read road 0 (always in bounds) and are masked
                const uint32_t idx = lane + (uint32_t)j * G;
                const bool ok = j < nslots && idx < deg;
                valid |= (ok ? 1u : 0u) << j;
                uint2 ph;
                if (pre) {
                    r0[j] = p0[j];
                    r1[j] = p1[j];
                    ph = pth[j];
                } else {
                    const uint32_t e = ok ? beg + idx : 0u;
                    const uint4* rp = reinterpret_cast<const uint4*>(a.rec + e);
                    r0[j] = __ldg(rp);
                    r1[j] = __ldg(rp + 1);
                    ph = __ldg(th + e);
                }
                tf[j] = ph.x ? __uint_as_float(ph.x) : base_tf;  // 0: the road still holds the baseline
                he[j] = ph.y;
            }
            // when any group of the warp has used up its buffered draws, every group refills from its
            // current step (lane l computes the draw of step + l), so refills stay rare and warp-wide
            if (__any_sync(FULL, stepping && (!rb_valid || steps - rb_base >= (uint32_t)G))) {
                const uint4 o = philox4x32_10(make_uint4(it, k, steps + lane, 0u), s0, s1);
                rb_x = o.x;
                rb_y = o.y;
                rb_base = steps;
                rb_valid = true;
            }
            const uint32_t rsrc = (steps - rb_base) & (uint32_t)(G - 1);
            const uint32_t rx = __shfl_sync(FULL, rb_x, rsrc, G), ry = __shfl_sync(FULL, rb_y, rsrc, G);
            const unsigned long long rnd = (unsigned long long)rx | ((unsigned long long)ry << 32);
            uint32_t cmask = 0, cong = 0;
            uint32_t sb[K], wv[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const uint32_t v = r0[j].x, cy = r1[j].x & kCycleMask;
                const bool unvisited = !((tabu[v >> 5] >> (v & 31)) & 1u);
                cmask |= ((valid >> j) & (unvisited ? 1u : 0u)) << j;
                cong |= (r0[j].w >> 31) << j;
                const uint32_t sw = signal_wait(a.t_dep + t + r0[j].z, cy | (cy == 0u), r1[j].w, r1[j].y, r1[j].z);
                const uint32_t w = (v != dst && cy != 0u) ? sw + (r0[j].w & kQdMask) : 0u;
                wv[j] = w;
                sb[j] = __float_as_uint(score_q(tf[j], alpha, reduced_cost(r0[j].z + w + he[j], hu), beta, frac));
            }
            constexpr uint32_t kGroupBits = G == 32 ? FULL : ((1u << (G & 31)) - 1u);
            const uint32_t gshift = wl & ~(uint32_t)(G - 1);
            if (a.thr_on) {  // congested roads drop out unless every candidate of the ant is congested
                const uint32_t g_ok = __ballot_sync(FULL, (cmask & ~cong) != 0u) >> gshift;
                const uint32_t g_cg = __ballot_sync(FULL, (cmask & cong) != 0u) >> gshift;
                if ((g_ok & kGroupBits) && (g_cg & kGroupBits)) cmask &= ~cong;
            }
            const bool has = ((__ballot_sync(FULL, cmask != 0u) >> gshift) & kGroupBits) != 0u;
            const bool back = stepping && !has && len > 0u;  // no way on: step back along the route
            if (stepping && !has && len == 0u) {              // back at src with no road left
                done = true;
                status = kAntDeadEnd;
            }
            // largest candidate score of each group, own weights, gather, roulette pick
            uint32_t mb = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) mb = max(mb, (cmask >> j & 1u) ? sb[j] : 0u);
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(FULL, mb, off, G));
            const WeightScale sc = weight_scale(mb);
            uint32_t incl[NC];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const uint32_t mine = (cmask >> j & 1u) ? roulette_weight_f(sb[j], sc) : 0u;
#pragma unroll
                for (int l = 0; l < G; ++l) incl[j * G + l] = j < nslots ? __shfl_sync(FULL, mine, l, G) : 0u;
            }
#pragma unroll
            for (int h = 1; h < NC; h <<= 1)
#pragma unroll
                for (int i = NC - 1; i >= h; --i) incl[i] += incl[i - h];
            const uint32_t r = draw_index(rnd, incl[NC - 1]);
            int pick = 0;
#pragma unroll
            for (int i = 0; i < NC; ++i) pick += incl[i] <= r ? 1 : 0;
            pick = min(pick, NC - 1);  // groups without candidates: any in-range slot (result unused)
            const int pick_lane = pick % G, pick_slot = pick / G;
            uint32_t c_h = 0, c_vb = 0, c_ve = 0, c_tt = 0, c_w = 0, c_he = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const bool sel = pick_slot == j;
                c_h = sel ? r0[j].x : c_h;
                c_vb = sel ? r0[j].y : c_vb;
                c_ve = sel ? r0[j].y + (r1[j].x >> 24) : c_ve;
                c_tt = sel ? r0[j].z : c_tt;
                c_w = sel ? wv[j] : c_w;
                c_he = sel ? he[j] : c_he;
            }
            c_h = __shfl_sync(FULL, c_h, pick_lane, G);
            c_vb = __shfl_sync(FULL, c_vb, pick_lane, G);
            c_ve = __shfl_sync(FULL, c_ve, pick_lane, G);
            c_tt = __shfl_sync(FULL, c_tt, pick_lane, G);
            c_w = __shfl_sync(FULL, c_w, pick_lane, G);
            c_he = __shfl_sync(FULL, c_he, pick_lane, G);
            if (back) {  // leave u (it stays visited, noted at the back of the route buffer) with its clock
                route[a.max_steps - 1u - pops] = u;  // every lane of the group, the same word
                ++pops;
                --len;
                const uint32_t e_in = route[len], w_in = rwait[len];
                t -= __ldg(&a.rec[e_in].tt) + w_in;
                W -= w_in;
                const StandPoint p = stand_after_back(a, th, route, len, src, qi);
                u = p.u;
                beg = p.beg;
                end = p.end;
                hu = p.h;
                ++steps;
            }
            if ((stepping && !done) || back) {
                if (!back) {
                    // every lane of the group writes the same words: no lane-dependent branch per step
                    route[len] = beg + (uint32_t)pick_lane + (uint32_t)pick_slot * G;
                    rwait[len] = c_w;
                    mark_visited(tabu, c_h);
                    t += c_tt + c_w;
                    W += c_w;
                    u = c_h;
                    beg = c_vb;
                    end = c_ve;
                    hu = c_he;
                    ++len;
                    ++steps;
                    if (t > kTCap) {
                        done = true;
                        status = kAntTimeCap;
                    }
                }
#pragma unroll
                for (int j = 0; j < K; ++j) {  // the rows of the next step, read past the masked slots as road 0
                    const uint32_t idx = lane + (uint32_t)j * G;
                    const uint32_t e = idx < end - beg ? beg + idx : 0u;
                    const uint4* rp = reinterpret_cast<const uint4*>(a.rec + e);
                    p0[j] = __ldg(rp);
                    p1[j] = __ldg(rp + 1);
                    pth[j] = __ldg(th + e);
                }
                pre = true;
            } else {
                pre = false;
            }
            __syncwarp();
        }
        // 3. ants that ended: the group records, deposits and resets its bitmap
        const bool any_done = __any_sync(FULL, done);
        want = want || any_done;
        if (any_done) {
            if (done) {
                QueryState* S = a.qs + qi;
                if (leader) {
                    a.ant_steps[slot] = len;
                    a.ant_wait[slot] = W;
                    atomicAdd(&S->steps, (unsigned long long)steps);
                    if (a.ant_log) {
                        uint32_t* l = a.ant_log + 4ull * (log_base + (uint64_t)it * n_ants + k);
                        *reinterpret_cast<uint4*>(l) = make_uint4(status | (len << 8), steps, t, W);
                    }
                }
                if (status == kAntSuccess) {  // Updt_Pher: deposit ant_deposit() on every road of the route
                    const unsigned long long delta = ant_deposit(S->dep_num, t);
                    unsigned long long* D = a.dep + (size_t)qi * a.n_edges;
                    for (uint32_t i = lane; i < len; i += G) {
                        atomicAdd(D + route[i], delta);
                        if (a.sparse) register_road(a, qi, S, route[i]);
                    }
                    if (leader) {
                        atomicAdd(&S->nsucc, 1ull);
                        atomicMin(&S->best_key, ((unsigned long long)t << 32) | ((unsigned long long)it * n_ants + k));
                    }
                }
                forget_visited(a, tabu, route, src, len, pops, steps, lane, G);
                active = false;
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Ant construction, one thread per ant, warp in lockstep. Every loop iteration the 32 ants of a warp
// take one step through the same branch-free code (K candidate slots per thread evaluated with
// instruction-level parallelism: independent loads and scores, then max, integer weights, running
// sum and the roulette pick in registers). Ants that end are finalised by the whole warp together
// (their deposits and their visited bitmap spread over 32 lanes), and the threads that became free
// take new ants with one warp-aggregated atomic. Visited bitmaps live in shared memory, word w of
// lane l at [w][l ^ (w mod 32)]: conflict-free both for one word of every lane and for every word of
// one lane.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tabu_index(uint32_t w, uint32_t l) { return w * 32u + ((l ^ w) & 31u); }

template <int K>
__global__ void __launch_bounds__(64) k_construct_lock(ConstructArgs a, uint32_t it) {
    extern __shared__ uint32_t smem[];
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t words = a.tabu_words;
    uint32_t* const tw = smem + (size_t)warp * words * 32u;  // this warp's bitmaps
    for (uint32_t w = lane; w < words * 32u; w += 32u) tw[w] = 0;
    __syncwarp();
    const uint32_t lt_mask = (1u << lane) - 1u;
    // per-thread ant
    bool active = false, exhausted = false, first = true;
    uint32_t qi = 0, k = 0, slot = 0, src = 0, dst = 0, n_ants = 1, alpha = 1, beta = 2, s0 = 0, s1 = 0;
    bool frac = false;  // non-integer exponents: alpha and beta are binary32 bits
    uint64_t log_base = 0;
    uint32_t u = 0, beg = 0, end = 0, t = 0, W = 0, steps = 0, status = 0;
    uint32_t len = 0, hu = 0;  // roads in the route, remaining bound at u
    const uint2* th = a.th;
    float base_tf = 0.0f;  // sparse layout: the colony's baseline pheromone of this iteration
    uint32_t* route = a.routes;
    uint32_t* rwait = a.rwait;
    const uint32_t n_threads = gridDim.x * blockDim.x;
    for (;;) {
        // 1. threads without an ant take the next ticket (the first one statically, no atomic)
        const bool need = !active && !exhausted;
        const uint32_t nmask = __ballot_sync(FULL, need);
        if (nmask) {
            uint32_t tk = blockIdx.x * blockDim.x + threadIdx.x;
            if (!first) {
                const int leader = __ffs(nmask) - 1;
                uint32_t base = 0;
                if ((int)lane == leader) base = atomicAdd(a.tickets + it, (uint32_t)__popc(nmask));
                base = __shfl_sync(FULL, base, leader);
                tk = n_threads + base + (uint32_t)__popc(nmask & lt_mask);
            }
            first = false;
            if (need) {
                if (tk >= a.total_ants) {
                    exhausted = true;
                } else {
                    const uint32_t tg = a.ticket_base + tk;  // the ant's index in the whole job
                    uint32_t lo = 0, hi = a.n_queries;  // query with ant_prefix[q] <= tg < ant_prefix[q + 1]
                    while (hi - lo > 1u) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (__ldg(a.ant_prefix + mid) <= tg) lo = mid;
                        else hi = mid;
                    }
                    const DevQuery q = a.queries[lo];
                    if (q.active && it < q.n_iter) {
                        active = true;
                        qi = lo;
                        k = tg - q.ant_base;
                        slot = tg;
                        src = q.src;
                        dst = q.dst;
                        n_ants = q.n_ants;
                        alpha = q.alpha;
                        beta = q.beta;
                        frac = (q.active & kQueryFracExp) != 0u;
                        s0 = (uint32_t)q.seed;
                        s1 = (uint32_t)(q.seed >> 32);
                        log_base = q.log_base;
                        th = a.th + (size_t)qi * a.n_edges;
                        base_tf = a.sparse ? __uint_as_float(a.qs[qi].base_tf) : 0.0f;
                        route = a.routes + (size_t)slot * a.max_steps;
                        rwait = a.rwait + (size_t)slot * a.max_steps;
                        u = src;
                        beg = __ldg(a.row_ptr + u);
                        end = __ldg(a.row_ptr + u + 1);
                        hu = a.qs[qi].h_src;
                        t = W = steps = len = 0;
                        tw[tabu_index(u >> 5, lane)] |= 1u << (u & 31);
                    }
                }
            }
        }
        if (!__any_sync(FULL, active || !exhausted)) break;
        if (!__any_sync(FULL, active)) continue;
        // 2. one step of every active ant
        bool done = false;
        if (active && u == dst) {
            done = true;
            status = kAntSuccess;
        } else if (active && steps == a.max_steps) {
            done = true;
            status = kAntStepCap;
        }
        const bool stepping = active && !done;
        const uint32_t deg = stepping ? end - beg : 0u;
        const uint32_t wmax = __reduce_max_sync(FULL, deg);
        uint32_t cmask = 0;  // candidates of this thread's ant (none when every row of the warp is empty)
        int js = 0;
        uint32_t c_h = 0, c_vb = 0, c_ve = 0, c_tt = 0, c_w = 0, c_he = 0;
        if (wmax > 0u) {
            uint4 r0[K], r1[K];
            float tf[K];
            uint32_t he[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if ((uint32_t)j < wmax) {  // warp-uniform; slots past a row read road 0 and are masked
                    const uint32_t e = (uint32_t)j < deg ? beg + j : 0u;
                    const uint4* rp = reinterpret_cast<const uint4*>(a.rec + e);
                    r0[j] = __ldg(rp);
                    r1[j] = __ldg(rp + 1);
                        const uint2 ph = __ldg(th + e);
                    tf[j] = ph.x ? __uint_as_float(ph.x) : base_tf;  // 0: the road still holds the baseline
                    he[j] = ph.y;
                } else {
                    r0[j] = r1[j] = make_uint4(0, 0, 0, 0);
                    tf[j] = 0.0f;
                    he[j] = 0;
                }
            }
            const uint4 o = philox4x32_10(make_uint4(it, k, steps, 0u), s0, s1);
            const unsigned long long rnd = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
            uint32_t cong = 0;
            uint32_t sb[K], wv[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                sb[j] = wv[j] = 0;
                if ((uint32_t)j < wmax) {
                    const uint32_t v = r0[j].x, cy = r1[j].x & kCycleMask;
                    const bool unvisited = !((tw[tabu_index(v >> 5, lane)] >> (v & 31)) & 1u);
                    cmask |= (((uint32_t)j < deg && unvisited) ? 1u : 0u) << j;
                    cong |= (r0[j].w >> 31) << j;
                    const uint32_t sw =
                        signal_wait(a.t_dep + t + r0[j].z, cy | (cy == 0u), r1[j].w, r1[j].y, r1[j].z);
                    const uint32_t w = (v != dst && cy != 0u) ? sw + (r0[j].w & kQdMask) : 0u;
                    wv[j] = w;
                    sb[j] = __float_as_uint(score_q(tf[j], alpha, reduced_cost(r0[j].z + w + he[j], hu), beta, frac));
                }
            }
            if (a.thr_on && (cmask & ~cong) && (cmask & cong)) cmask &= ~cong;
            uint32_t mb = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) mb = max(mb, (cmask >> j & 1u) ? sb[j] : 0u);
            const WeightScale sc = weight_scale(mb);
            uint32_t incl[K], S = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                S += (cmask >> j & 1u) ? roulette_weight_f(sb[j], sc) : 0u;
                incl[j] = S;
            }
            const uint32_t r = draw_index(rnd, S);
            bool found = false;
#pragma unroll
            for (int j = 0; j < K; ++j) {  // first candidate whose running weight exceeds r
                const bool hit = !found && (cmask >> j & 1u) && incl[j] > r;
                js = hit ? j : js;
                found |= hit;
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const bool sel = js == j;
                c_h = sel ? r0[j].x : c_h;
                c_vb = sel ? r0[j].y : c_vb;
                c_ve = sel ? r0[j].y + (r1[j].x >> 24) : c_ve;
                c_tt = sel ? r0[j].z : c_tt;
                c_w = sel ? wv[j] : c_w;
                c_he = sel ? he[j] : c_he;
            }
        }
        if (stepping && cmask == 0u) {
            if (len == 0u) {  // back at src with no road left
                done = true;
                status = kAntDeadEnd;
            } else {  // step back along the route with the clock it had there (u stays visited)
                --len;
                const uint32_t e_in = route[len], w_in = rwait[len];
                t -= __ldg(&a.rec[e_in].tt) + w_in;
                W -= w_in;
                const StandPoint p = stand_after_back(a, th, route, len, src, qi);
                u = p.u;
                beg = p.beg;
                end = p.end;
                hu = p.h;
                ++steps;
            }
        } else if (stepping) {
            route[len] = beg + (uint32_t)js;
            rwait[len] = c_w;
            t += c_tt + c_w;
            W += c_w;
            u = c_h;
            beg = c_vb;
            end = c_ve;
            hu = c_he;
            tw[tabu_index(u >> 5, lane)] |= 1u << (u & 31);
            ++len;
            ++steps;
            if (t > kTCap) {
                done = true;
                status = kAntTimeCap;
            }
        }
        // 3. ants that ended: per-ant records by their own lane, deposits and bitmap reset by the warp
        uint32_t fmask = __ballot_sync(FULL, done);
        if (fmask) {
            unsigned long long delta = 0;
            if (done) {
                QueryState* S = a.qs + qi;
                a.ant_steps[slot] = len;
                a.ant_wait[slot] = W;
                atomicAdd(&S->steps, (unsigned long long)steps);
                if (a.ant_log) {
                    uint32_t* l = a.ant_log + 4ull * (log_base + (uint64_t)it * n_ants + k);
                    *reinterpret_cast<uint4*>(l) = make_uint4(status | (len << 8), steps, t, W);
                }
                if (status == kAntSuccess) {
                    atomicAdd(&S->nsucc, 1ull);
                    delta = ant_deposit(S->dep_num, t);
                    atomicMin(&S->best_key, ((unsigned long long)t << 32) | ((unsigned long long)it * n_ants + k));
                }
            }
            __syncwarp();
            while (fmask) {
                const int f = __ffs(fmask) - 1;
                fmask &= fmask - 1u;
                const unsigned long long fd = __shfl_sync(FULL, delta, f);
                const uint32_t fsteps = __shfl_sync(FULL, len, f);
                const uint32_t fqi = __shfl_sync(FULL, qi, f);
                const uint32_t fslot = __shfl_sync(FULL, slot, f);
                if (fd) {  // Updt_Pher: deposit ant_deposit() on every road of the route
                    unsigned long long* D = a.dep + (size_t)fqi * a.n_edges;
                    const uint32_t* fr = a.routes + (size_t)fslot * a.max_steps;
                    for (uint32_t i = lane; i < fsteps; i += 32u) {
                        atomicAdd(D + fr[i], fd);
                        if (a.sparse) register_road(a, fqi, a.qs + fqi, fr[i]);
                    }
                }
                for (uint32_t w = lane; w < words; w += 32u) tw[tabu_index(w, (uint32_t)f)] = 0;
            }
            __syncwarp();
            if (done) active = false;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Evap_Pher + Updt_Pher: tau <- tau - floor(tau * rho_fix / 2^32) + D ; D <- 0 (tau_next).
// ------------------------------------------------------------------------------------------------
// Iteration end, one launch for three independent pieces of work (all read what the construction
// kernel wrote, none reads what another writes):
//   Evap_Pher + Updt_Pher  tau <- tau - floor(tau * rho_fix / 2^32) + D, D <- 0, per (colony, road)
//                          (under GMP_FLAG_EVAP_UNUSED a road with D > 0 keeps tau + D), then the
//                          road's binary32 pheromone word (tau_word);
//   best-route tracking    when a colony's best key came from this iteration, keep that ant's route;
//   Calc_Dens / Comp_Thres the per-intersection phase order (densities are fixed within a job, so the
//                          update reproduces the same order; it runs because the iteration calls it).
// Blocks [0, nev) evaporate kEvapPer roads per thread with every load issued first; the next Q blocks
// copy best routes; the rest update intersections.
constexpr uint32_t kEvapPer = 4;
constexpr uint32_t kSparseEvapBlocks = 8;
constexpr uint32_t kIterEndBlock = 256;

__global__ void __launch_bounds__(kIterEndBlock) k_iter_end(IterEndArgs a) {
    uint32_t b = blockIdx.x;
    const uint32_t nev = a.n_queries * a.evap_blocks;
    if (b < nev) {
        const uint32_t qi = b / a.evap_blocks, chunk = b - qi * a.evap_blocks;
        const DevQuery& Q = a.q[qi];
        if (!Q.active || a.it >= Q.n_iter) return;
        const uint64_t rf = Q.rho_fix;
        const size_t off = (size_t)qi * a.n_edges;
        if (a.sparse) {  // only the roads with deposits so far hold their own pheromone
            const uint32_t n = a.qs[qi].n_touched;
            const uint32_t* LE = a.list_e + off;
            uint64_t* LT = a.list_tau + off;
            unsigned long long* D = a.dep + off;
            uint32_t* TF = reinterpret_cast<uint32_t*>(a.th + off);
            for (uint32_t i = chunk * kIterEndBlock + threadIdx.x; i < n; i += a.evap_blocks * kIterEndBlock) {
                const uint32_t e = LE[i];
                const uint64_t nt = tau_next(LT[i], rf, D[e], a.flags);
                LT[i] = nt;
                D[e] = 0;
                TF[2 * (size_t)e] = tau_word(nt, a.flags);
            }
            return;
        }
        uint64_t* T = a.tau + off;
        uint32_t* TF = reinterpret_cast<uint32_t*>(a.th + off);  // pheromone half of each pair
        unsigned long long* D = a.dep + off;
        const uint32_t e0 = chunk * kIterEndBlock * kEvapPer + threadIdx.x;
        uint64_t tv[kEvapPer];
        unsigned long long dv[kEvapPer];
#pragma unroll
        for (uint32_t i = 0; i < kEvapPer; ++i) {
            const uint32_t e = e0 + i * kIterEndBlock;
            tv[i] = e < a.n_edges ? T[e] : 0;
            dv[i] = e < a.n_edges ? D[e] : 0;
        }
#pragma unroll
        for (uint32_t i = 0; i < kEvapPer; ++i) {
            const uint32_t e = e0 + i * kIterEndBlock;
            if (e < a.n_edges) {
                const uint64_t nt = tau_next(tv[i], rf, dv[i], a.flags);
                T[e] = nt;
                TF[2 * (size_t)e] = tau_word(nt, a.flags);
                D[e] = 0;
            }
        }
        return;
    }
    b -= nev;
    if (b < a.n_queries) {
        const uint32_t qi = b;
        const DevQuery Q = a.q[qi];
        if (!Q.active || a.it >= Q.n_iter) return;
        if (a.sparse && threadIdx.x == 0) {  // the baseline: every road without a deposit evaporates alike
            const uint64_t nt = tau_next(a.qs[qi].base_tau, Q.rho_fix, 0, a.flags);
            a.qs[qi].base_tau = nt;
            a.qs[qi].base_tf = tau_word(nt, a.flags);
        }
        const unsigned long long key = a.qs[qi].best_key;
        if (key == kNoKey) return;
        const uint32_t low = (uint32_t)key;
        if (low / Q.n_ants != a.it) return;
        const uint32_t slot = Q.ant_base + low % Q.n_ants;
        const uint32_t len = a.ant_steps[slot];
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
            a.best_route[(size_t)qi * a.max_steps + i] = a.routes[(size_t)slot * a.max_steps + i];
        if (threadIdx.x == 0) {
            a.qs[qi].best_len = len;
            a.qs[qi].best_W = a.ant_wait[slot];
        }
        return;
    }
    b -= a.n_queries;
    const uint32_t v = b * blockDim.x + threadIdx.x;
    if (v < a.n_nodes)  // intersections with more than two phases: a separate launch (k_queue_general)
        queue_node_small<false, false>(v, a.qt);
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

cudaError_t launch_edge_static(cudaStream_t s, uint32_t E, const uint32_t* in_edge, const uint32_t* len,
                               const uint16_t* speed, const uint8_t* lanes_by_road, uint32_t* ff, uint32_t* cap,
                               uint8_t* lanes) {
    if (E == 0) return cudaSuccess;
    k_edge_static<<<blocks_for(E, 256), 256, 0, s>>>(E, in_edge, len, speed, lanes_by_road, ff, cap, lanes);
    return cudaGetLastError();
}

cudaError_t launch_gather_u32(cudaStream_t s, uint32_t n, const uint32_t* idx, const uint32_t* src, uint32_t* dst) {
    if (n == 0) return cudaSuccess;
    k_gather<uint32_t><<<blocks_for(n, 256), 256, 0, s>>>(n, idx, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_gather_u8(cudaStream_t s, uint32_t n, const uint32_t* idx, const uint8_t* src, uint8_t* dst) {
    if (n == 0) return cudaSuccess;
    k_gather<uint8_t><<<blocks_for(n, 256), 256, 0, s>>>(n, idx, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_queue_general(cudaStream_t s, const QueueTables& t, QueuePass pass) {
    if (t.n_nodes == 0) return cudaSuccess;
    const unsigned g = blocks_for(t.n_nodes, 128);
    if (pass == QueuePass::kRefresh) k_queue_general<true, false><<<g, 128, 0, s>>>(t);
    else if (pass == QueuePass::kTick) k_queue_general<true, true><<<g, 128, 0, s>>>(t);
    else k_queue_general<false, false><<<g, 128, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_queue(cudaStream_t s, const QueueTables& t, uint32_t max_phases, QueuePass pass) {
    if (t.n_nodes == 0) return cudaSuccess;
    const unsigned g = blocks_for(t.n_nodes, 128);
    if (pass == QueuePass::kRefresh) k_queue_small<true, false><<<g, 128, 0, s>>>(t);
    else if (pass == QueuePass::kTick) k_queue_small<true, true><<<g, 128, 0, s>>>(t);
    else k_queue_small<false, false><<<g, 128, 0, s>>>(t);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && max_phases > 2) err = launch_queue_general(s, t, pass);
    return err;
}

cudaError_t launch_tick_node(cudaStream_t s, const QueueTables& t, uint64_t t_now, uint32_t dt,
                             uint32_t red_planes, uint32_t* leave, unsigned long long* K) {
    if (t.n_nodes == 0) return cudaSuccess;
    TickCap tc;
    for (uint32_t L = 0; L < 256; ++L) {
        const uint64_t c = (uint64_t)L * (t_now + dt) / t.h_sat - (uint64_t)L * t_now / t.h_sat;
        tc.cap[L] = c > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)c;
    }
    k_tick_node<<<blocks_for(t.n_nodes, 128), 128, 0, s>>>(t, t_now, dt, red_planes, tc, leave, K);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(cudaStream_t s, uint32_t Q, uint32_t E, const DevQuery* q, const uint32_t* col,
                              const int32_t* x, const int32_t* y, uint32_t kappa, uint32_t flags, uint64_t* tau,
                              uint2* th, unsigned long long* dep, QueryState* qs, uint32_t* tickets,
                              uint32_t n_tickets, uint32_t sparse, uint32_t* tflag, uint32_t tflag_words,
                              const uint32_t* hdist, uint32_t N, bool zero_dep) {
    if (Q == 0) return cudaSuccess;
    dim3 grid(blocks_for(E ? E : 1, 256), (Q + kInitCols - 1) / kInitCols);
#define GMP_INIT(EX_, REP_)                                                                                 \
    k_init_batch<EX_, REP_><<<grid, 256, 0, s>>>(Q, E, q, col, x, y, kappa, flags, tau, th, dep, qs, tickets, n_tickets, \
                                                 sparse, tflag, tflag_words, hdist, N, zero_dep ? 1u : 0u)
    const bool rep = (flags & GMP_FLAG_REPULSIVE) != 0;
    if (hdist) {
        if (rep) GMP_INIT(true, true);
        else GMP_INIT(true, false);
    } else {
        if (rep) GMP_INIT(false, true);
        else GMP_INIT(false, false);
    }
#undef GMP_INIT
    return cudaGetLastError();
}

cudaError_t launch_exact_h(cudaStream_t s, uint32_t Q, uint32_t N, const DevQuery* q, const uint32_t* in_ptr,
                           const uint32_t* in_edge, const uint32_t* in_tail, const EdgeRec* rec, uint32_t delta,
                           uint32_t level_limit, uint32_t* hdist, uint32_t* queue, uint32_t* stamps, uint32_t* err) {
    if (Q == 0 || N == 0) return cudaSuccess;
    k_exact_h<<<Q, kExactHBlock, 0, s>>>(N, q, in_ptr, in_edge, in_tail, rec, delta, level_limit, hdist, queue,
                                         stamps, err);
    return cudaGetLastError();
}

cudaError_t launch_iter_end(cudaStream_t s, const IterEndArgs& args) {
    IterEndArgs a = args;
    a.evap_blocks = (a.n_edges + kIterEndBlock * kEvapPer - 1) / (kIterEndBlock * kEvapPer);
    // sparse layout: a few blocks per colony stride over its registered roads (far fewer than E)
    if (a.sparse && a.evap_blocks > kSparseEvapBlocks) a.evap_blocks = kSparseEvapBlocks;
    const uint64_t blocks = (uint64_t)a.n_queries * a.evap_blocks + a.n_queries +
                            (a.n_nodes + kIterEndBlock - 1) / kIterEndBlock;
    if (blocks == 0) return cudaSuccess;
    k_iter_end<<<(uint32_t)blocks, kIterEndBlock, 0, s>>>(a);
    return cudaGetLastError();
}

// Dense pheromone of one colony from the sparse layout: the baseline everywhere, then the registered
// roads' own values (for reading the table back).
__global__ void k_materialize_tau(uint32_t E, const QueryState* __restrict__ qs, const uint32_t* __restrict__ list_e,
                                  const uint64_t* __restrict__ list_tau, uint64_t* __restrict__ out, uint32_t phase) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (phase == 0) {
        if (i < E) out[i] = qs->base_tau;
    } else if (i < qs->n_touched) {
        out[list_e[i]] = list_tau[i];
    }
}

cudaError_t launch_materialize_tau(cudaStream_t s, uint32_t E, const QueryState* qs, const uint32_t* list_e,
                                   const uint64_t* list_tau, uint64_t* out) {
    if (E == 0) return cudaSuccess;
    k_materialize_tau<<<blocks_for(E, 256), 256, 0, s>>>(E, qs, list_e, list_tau, out, 0);
    k_materialize_tau<<<blocks_for(E, 256), 256, 0, s>>>(E, qs, list_e, list_tau, out, 1);
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
    int per_sm = 0, sms = 0;
    if (in_smem) {
        if (dyn > 48u * 1024u) {
            // per kernel function, shared by every context: the cap of in-smem bitmaps, not this size
            err = cudaFuncSetAttribute(k_construct<G, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       64 * 1024);
            if (err != cudaSuccess) return err;
        }
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct<G, K, true>, block, dyn);
    } else {
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct<G, K, false>, block, 0);
    }
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

int construct_max_degree(int lanes) { return lanes == 1 ? 8 : lanes * 4; }

// Lockstep thread-per-ant variant: visited bitmaps of every thread of the block in shared memory.
template <int K>
static cudaError_t config_t(int device, uint32_t n_nodes, uint32_t total_ants, KernelConfig* out) {
    const int block = 64;
    const uint32_t words = (n_nodes + 31u) / 32u;
    const size_t smem = (size_t)block * words * 4u;
    if (smem > 200u * 1024u) return cudaErrorInvalidValue;
    cudaError_t err;
    if (smem > 48u * 1024u) {
        // per kernel function, shared by every context: the cap of this kernel's bitmaps, not this size
        err = cudaFuncSetAttribute(k_construct_lock<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (err != cudaSuccess) return err;
    }
    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct_lock<K>, block, smem);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidValue;
    const uint64_t need = ((uint64_t)total_ants + block - 1) / block;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (need < grid) grid = need;
    out->lanes = 1;
    out->slots = K;
    out->block = block;
    out->grid = (int)(grid < 1 ? 1 : grid);
    out->smem = smem;
    out->tabu_in_smem = true;
    out->lockstep = false;  // dispatched on lanes == 1
    return cudaSuccess;
}

bool construct_thread_fits(uint32_t n_nodes) { return 64ull * ((n_nodes + 31u) / 32u) * 4u <= 200u * 1024u; }

cudaError_t construct_config(int device, int lanes, uint32_t n_nodes, uint32_t max_degree, uint32_t total_ants,
                             KernelConfig* out) {
    if (lanes == 1) {
        if (max_degree <= 4) return config_t<4>(device, n_nodes, total_ants, out);
        if (max_degree <= 6) return config_t<6>(device, n_nodes, total_ants, out);
        if (max_degree <= 8) return config_t<8>(device, n_nodes, total_ants, out);
        return cudaErrorInvalidValue;
    }
    const int k = slots_for(lanes, max_degree);
#define GMP_CFG(G_, K_) \
    if (lanes == G_ && k == K_) return config_for<G_, K_>(device, n_nodes, total_ants, out);
    GMP_CFG(4, 1) GMP_CFG(4, 2) GMP_CFG(4, 4) GMP_CFG(8, 1) GMP_CFG(8, 2) GMP_CFG(8, 4)
    GMP_CFG(16, 1) GMP_CFG(16, 2) GMP_CFG(16, 4) GMP_CFG(32, 1) GMP_CFG(32, 2) GMP_CFG(32, 4)
#undef GMP_CFG
    return cudaErrorInvalidValue;
}

template <int G, int K>
static cudaError_t config_gl(int device, uint32_t n_nodes, uint32_t total_ants, bool frac, KernelConfig* out) {
    const int block = 128;
    const int groups = block / G;
    const uint32_t words = (n_nodes + 31u) / 32u;
    const size_t smem = (size_t)groups * words * 4u;
    const bool in_smem = smem <= 64u * 1024u;
    const size_t dyn = in_smem ? smem : 0;
    cudaError_t err;
    int per_sm = 0, sms = 0;
    if (in_smem) {
        if (dyn > 48u * 1024u) {
            // per kernel function, shared by every context: the cap of in-smem bitmaps, not this size
            err = cudaFuncSetAttribute(k_construct_gl<G, K, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       64 * 1024);
            if (err == cudaSuccess)
                err = cudaFuncSetAttribute(k_construct_gl<G, K, true, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
            if (err != cudaSuccess) return err;
        }
        err = frac ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct_gl<G, K, true, true>, block, dyn)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct_gl<G, K, true, false>, block,
                                                                   dyn);
    } else {
        err = frac ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct_gl<G, K, false, true>, block, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_construct_gl<G, K, false, false>, block,
                                                                   0);
    }
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    const uint64_t need = ((uint64_t)total_ants + groups - 1) / groups;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (need < grid) grid = need;
    out->lanes = G;
    out->slots = K;
    out->block = block;
    out->grid = (int)(grid < 1 ? 1 : grid);
    out->smem = dyn;
    out->tabu_in_smem = in_smem;
    out->lockstep = true;
    out->frac = frac;
    return cudaSuccess;
}

cudaError_t construct_config_lockstep(int device, int lanes, uint32_t n_nodes, uint32_t max_degree,
                                      uint32_t total_ants, bool frac, KernelConfig* out) {
    const int k = (uint32_t)lanes >= max_degree ? 1 : ((uint32_t)(2 * lanes) >= max_degree ? 2 : 0);
    if (lanes == 4 && k == 1) return config_gl<4, 1>(device, n_nodes, total_ants, frac, out);
    if (lanes == 4 && k == 2) return config_gl<4, 2>(device, n_nodes, total_ants, frac, out);
    if (lanes == 8 && k == 1) return config_gl<8, 1>(device, n_nodes, total_ants, frac, out);
    if (lanes == 8 && k == 2) return config_gl<8, 2>(device, n_nodes, total_ants, frac, out);
    if (lanes == 16 && k == 1) return config_gl<16, 1>(device, n_nodes, total_ants, frac, out);
    return cudaErrorInvalidValue;
}

cudaError_t construct_tail_config(int device, uint32_t n_nodes, uint32_t total_ants, KernelConfig* out) {
    KernelConfig kc{};
    kc.lanes = 32;
    kc.slots = 1;
    kc.block = 128;
    kc.tabu_in_smem = true;
    kc.smem = (size_t)(kc.block / 32) * ((n_nodes + 31u) / 32u) * 4u;
    cudaError_t err = cudaSuccess;
    if (kc.smem > 48u * 1024u)
        err = cudaFuncSetAttribute(k_construct_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kc.smem);
    if (err != cudaSuccess) return err;
    // suspended walks are a few of the launch's ants: a modest grid whose warps loop over them
    const uint32_t warps = total_ants < 256u ? total_ants : 256u;
    kc.grid = (int)((warps + 3u) / 4u);
    if (kc.grid < 1) kc.grid = 1;
    (void)device;
    *out = kc;
    return cudaSuccess;
}

cudaError_t launch_construct_tail(cudaStream_t s, const KernelConfig& kc, const ConstructArgs& a, uint32_t it) {
    k_construct_tail<<<kc.grid, kc.block, kc.smem, s>>>(a, it);
    return cudaGetLastError();
}

cudaError_t launch_construct(cudaStream_t s, const KernelConfig& kc, const ConstructArgs& a, uint32_t it) {
    if (kc.lockstep) {
#define GMP_LAUNCH_GL(G_, K_)                                                                            \
    if (kc.lanes == G_ && kc.slots == K_) {                                                              \
        if (kc.frac) {                                                                                   \
            if (kc.tabu_in_smem) k_construct_gl<G_, K_, true, true><<<kc.grid, kc.block, kc.smem, s>>>(a, it); \
            else k_construct_gl<G_, K_, false, true><<<kc.grid, kc.block, 0, s>>>(a, it);               \
        } else {                                                                                         \
            if (kc.tabu_in_smem) k_construct_gl<G_, K_, true, false><<<kc.grid, kc.block, kc.smem, s>>>(a, it); \
            else k_construct_gl<G_, K_, false, false><<<kc.grid, kc.block, 0, s>>>(a, it);              \
        }                                                                                                \
        return cudaGetLastError();                                                                       \
    }
        GMP_LAUNCH_GL(4, 1) GMP_LAUNCH_GL(4, 2) GMP_LAUNCH_GL(8, 1) GMP_LAUNCH_GL(8, 2) GMP_LAUNCH_GL(16, 1)
#undef GMP_LAUNCH_GL
        return cudaErrorInvalidValue;
    }
#define GMP_LAUNCH(G_, K_)                                                            \
    if (kc.lanes == G_ && kc.slots == K_) {                                           \
        if (kc.tabu_in_smem) k_construct<G_, K_, true><<<kc.grid, kc.block, kc.smem, s>>>(a, it); \
        else k_construct<G_, K_, false><<<kc.grid, kc.block, 0, s>>>(a, it);          \
        return cudaGetLastError();                                                    \
    }
    if (kc.lanes == 1) {
        if (kc.slots == 4) k_construct_lock<4><<<kc.grid, kc.block, kc.smem, s>>>(a, it);
        else if (kc.slots == 6) k_construct_lock<6><<<kc.grid, kc.block, kc.smem, s>>>(a, it);
        else if (kc.slots == 8) k_construct_lock<8><<<kc.grid, kc.block, kc.smem, s>>>(a, it);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    GMP_LAUNCH(4, 1) GMP_LAUNCH(4, 2) GMP_LAUNCH(4, 4) GMP_LAUNCH(8, 1) GMP_LAUNCH(8, 2) GMP_LAUNCH(8, 4)
    GMP_LAUNCH(16, 1) GMP_LAUNCH(16, 2) GMP_LAUNCH(16, 4) GMP_LAUNCH(32, 1) GMP_LAUNCH(32, 2) GMP_LAUNCH(32, 4)
#undef GMP_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace gmp

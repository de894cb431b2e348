// Device routines shared by the iteration kernels (gmp_kernels.cu) and the persistent job
// (gmp_persistent.cu): the sub-warp ant walk and the preemptive phase order of one intersection.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp_device.cuh"
#include "gmp_internal.h"

namespace gmp {

// Preemptive phase order of intersection v (Calc_Dens / Comp_Thres; Fig. 3 signal block): queues and
// storage per phase from the node's in-edges; order (1) phases whose queue exceeds 3/4 of their
// storage, longest first; else (2) phases red for longer than a cycle, longest first; else (3) the
// longest non-empty queue; then the remaining non-empty phases, then the empty ones, each in index
// order. Every in-edge's record then gets its approach's green window under that order.
__device__ __forceinline__ void queue_node(uint32_t v, const uint32_t* __restrict__ row_ptr,
                                           const uint32_t* __restrict__ in_ptr,
                                           const uint32_t* __restrict__ in_edge, const uint8_t* __restrict__ nph,
                                           const uint32_t* __restrict__ cycle, const uint32_t* __restrict__ offset,
                                           const uint32_t* __restrict__ green, const uint8_t* __restrict__ ephase,
                                           const uint32_t* __restrict__ veh, const uint32_t* __restrict__ cap,
                                           const uint32_t* __restrict__ red, uint8_t* __restrict__ order,
                                           EdgeRec* __restrict__ rec) {
    const uint32_t P = nph[v], ib = in_ptr[v], ie = in_ptr[v + 1];
    const uint32_t deg = min(row_ptr[v + 1] - row_ptr[v], 255u) << 24;  // out-degree of v (at most 128 runs)
    if (P == 0) {
        for (uint32_t i = 0; i < kMaxPhases; ++i) order[(size_t)v * kMaxPhases + i] = (uint8_t)i;
        for (uint32_t i = ib; i < ie; ++i)  // second half of the record (see EdgeRec)
            reinterpret_cast<uint4*>(rec + in_edge[i])[1] = make_uint4(deg, 0u, 0u, 0u);
        return;
    }
    // everything below stays in registers: phase-indexed values are only read and written at
    // compile-time indices (loops over the 8 possible phases are unrolled and masked)
    uint64_t Q[kMaxPhases], S[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) Q[k] = S[k] = 0;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t e = in_edge[i];
        const uint32_t p = ephase[e] & (kMaxPhases - 1);
        const uint32_t n = veh[e], c = cap[e];
#pragma unroll
        for (uint32_t k = 0; k < kMaxPhases; ++k) {
            Q[k] += p == k ? n : 0u;
            S[k] += p == k ? c : 0u;
        }
    }
    const uint32_t cy = cycle[v];
    uint32_t over = 0, starved = 0, nonempty = 0;
    uint32_t rd[kMaxPhases], gr[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        rd[k] = k < P ? red[(size_t)v * kMaxPhases + k] : 0u;
        gr[k] = k < P ? green[(size_t)v * kMaxPhases + k] : 0u;
        if (k < P) {
            if (Q[k] > S[k] * 3u / 4u) over |= 1u << k;
            if (rd[k] > cy) starved |= 1u << k;
            if (Q[k] > 0) nonempty |= 1u << k;
        }
    }
    // the phases that go first, with the value that orders them (longest first, then lower index)
    uint32_t prio = 0;
    bool by_q = true;
    if (over) {
        prio = over;
    } else if (starved) {
        prio = starved;
        by_q = false;
    } else if (nonempty) {  // the longest non-empty queue (first in index order on ties)
        int best = -1;
        uint64_t bq = 0;
#pragma unroll
        for (uint32_t k = 0; k < kMaxPhases; ++k)
            if ((nonempty >> k & 1u) && (best < 0 || Q[k] > bq)) {
                best = (int)k;
                bq = Q[k];
            }
        prio = 1u << best;
    }
    // sort key per phase: prioritised phases by value descending, then the other non-empty phases, then
    // the empty ones, each in index order; the position of a phase in the plan is its rank by key
    constexpr uint64_t kVmax = (1ull << 48) - 1;
    uint64_t key[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        const uint64_t val = by_q ? Q[k] : (uint64_t)rd[k];
        const uint64_t grp = (prio >> k & 1u) ? 0u : ((nonempty >> k & 1u) ? 1u : 2u);
        key[k] = (grp << 60) | (grp == 0 ? (kVmax - (val < kVmax ? val : kVmax)) << 4 : 0u) | k;
    }
    uint32_t start[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        uint32_t rank = 0, st = 0;
#pragma unroll
        for (uint32_t q = 0; q < kMaxPhases; ++q)
            if (q < P && key[q] < key[k]) {
                ++rank;
                st += gr[q];
            }
        start[k] = st;
        if (k < P) order[(size_t)v * kMaxPhases + rank] = (uint8_t)k;
        else order[(size_t)v * kMaxPhases + k] = (uint8_t)k;
    }
    const uint32_t off = offset[v];
    const uint32_t magic = 0xFFFFFFFFu / cy;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t e = in_edge[i];
        const uint32_t p = ephase[e] & (kMaxPhases - 1);
        uint32_t st = 0, gl = 0;
#pragma unroll
        for (uint32_t k = 0; k < kMaxPhases; ++k) {
            st = p == k ? start[k] : st;
            gl = p == k ? gr[k] : gl;
        }
        reinterpret_cast<uint4*>(rec + e)[1] = make_uint4(cy | deg, (off + st) % cy, gl, magic);
    }
}

// queue_node for a node with at most two phases (unsignalised nodes, and every junction the generators
// build), with the same results in far fewer registers: two keys decide the whole order. Returns false,
// doing nothing, for a node with more phases (queue_node handles those). Phase p of a road into a
// signalised node is below its phase count and the greens add up to the cycle (both checked when the
// signals are set), so only phases 0 and 1 occur here.
__device__ __forceinline__ bool queue_node_small(uint32_t v, const uint32_t* __restrict__ row_ptr,
                                                 const uint32_t* __restrict__ in_ptr,
                                                 const uint32_t* __restrict__ in_edge, const uint8_t* __restrict__ nph,
                                                 const uint32_t* __restrict__ cycle,
                                                 const uint32_t* __restrict__ offset,
                                                 const uint32_t* __restrict__ green,
                                                 const uint8_t* __restrict__ ephase,
                                                 const uint32_t* __restrict__ veh, const uint32_t* __restrict__ cap,
                                                 const uint32_t* __restrict__ red, uint8_t* __restrict__ order,
                                                 EdgeRec* __restrict__ rec) {
    const uint32_t P = nph[v];
    if (P > 2) return false;
    const uint32_t ib = in_ptr[v], ie = in_ptr[v + 1];
    const uint32_t deg = min(row_ptr[v + 1] - row_ptr[v], 255u) << 24;  // out-degree of v (at most 128 runs)
    uint2* const ord = reinterpret_cast<uint2*>(order + (size_t)v * kMaxPhases);
    if (P == 0) {
        *ord = make_uint2(0x03020100u, 0x07060504u);  // identity order
        for (uint32_t i = ib; i < ie; ++i)  // second half of the record (see EdgeRec)
            reinterpret_cast<uint4*>(rec + in_edge[i])[1] = make_uint4(deg, 0u, 0u, 0u);
        return true;
    }
    uint64_t Q0 = 0, Q1 = 0, S0 = 0, S1 = 0;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t e = in_edge[i];
        const bool p1 = (ephase[e] & (kMaxPhases - 1)) != 0u;
        const uint32_t n = veh[e], c = cap[e];
        Q0 += p1 ? 0u : n;
        S0 += p1 ? 0u : c;
        Q1 += p1 ? n : 0u;
        S1 += p1 ? c : 0u;
    }
    const uint32_t cy = cycle[v];
    const uint32_t rd0 = red[(size_t)v * kMaxPhases], g0 = green[(size_t)v * kMaxPhases];
    const uint32_t rd1 = P > 1 ? red[(size_t)v * kMaxPhases + 1] : 0u;
    const uint32_t g1 = P > 1 ? green[(size_t)v * kMaxPhases + 1] : 0u;
    const uint32_t valid = P > 1 ? 3u : 1u;
    const uint32_t over = ((Q0 > S0 * 3u / 4u ? 1u : 0u) | (Q1 > S1 * 3u / 4u ? 2u : 0u)) & valid;
    const uint32_t starved = ((rd0 > cy ? 1u : 0u) | (rd1 > cy ? 2u : 0u)) & valid;
    const uint32_t nonempty = ((Q0 > 0 ? 1u : 0u) | (Q1 > 0 ? 2u : 0u)) & valid;
    uint32_t prio = 0;
    bool by_q = true;
    if (over) {
        prio = over;
    } else if (starved) {
        prio = starved;
        by_q = false;
    } else if (nonempty) {  // the longest non-empty queue, phase 0 on ties
        prio = ((nonempty & 1u) && (!(nonempty & 2u) || Q0 >= Q1)) ? 1u : 2u;
    }
    // the sort keys of queue_node; phase 0 goes first when its key is the smaller one
    constexpr uint64_t kVmax = (1ull << 48) - 1;
    const uint64_t v0 = by_q ? Q0 : (uint64_t)rd0, v1 = by_q ? Q1 : (uint64_t)rd1;
    const uint64_t grp0 = (prio & 1u) ? 0u : ((nonempty & 1u) ? 1u : 2u);
    const uint64_t grp1 = (prio & 2u) ? 0u : ((nonempty & 2u) ? 1u : 2u);
    const uint64_t key0 = (grp0 << 60) | (grp0 == 0 ? (kVmax - (v0 < kVmax ? v0 : kVmax)) << 4 : 0u);
    const uint64_t key1 = (grp1 << 60) | (grp1 == 0 ? (kVmax - (v1 < kVmax ? v1 : kVmax)) << 4 : 0u) | 1u;
    const bool first0 = P == 1 || key0 < key1;
    *ord = make_uint2(first0 ? 0x03020100u : 0x03020001u, 0x07060504u);
    const uint32_t st0 = first0 ? 0u : g1, st1 = first0 ? g0 : 0u;  // green-window starts in plan order
    const uint32_t off = offset[v];
    const uint32_t magic = 0xFFFFFFFFu / cy;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t e = in_edge[i];
        const bool p1 = (ephase[e] & (kMaxPhases - 1)) != 0u;
        reinterpret_cast<uint4*>(rec + e)[1] =
            make_uint4(cy | deg, (off + (p1 ? st1 : st0)) % cy, p1 ? g1 : g0, magic);
    }
    return true;
}

// Sparse pheromone layout: a road's first deposit of the job registers it in its colony's list,
// with the pheromone it held until then (the colony's baseline of this iteration); from then on the
// iteration end evaporates it on its own. The flag test before the atomic skips registered roads.
__device__ __forceinline__ void register_road(const ConstructArgs& a, uint32_t qi, QueryState* S, uint32_t e) {
    uint32_t* F = a.tflag + (size_t)qi * a.tflag_words + (e >> 5);
    const uint32_t bit = 1u << (e & 31);
    if (*(volatile const uint32_t*)F & bit) return;
    if (atomicOr(F, bit) & bit) return;
    const uint32_t idx = atomicAdd(&S->n_touched, 1u);
    a.list_e[(size_t)qi * a.n_edges + idx] = e;
    a.list_tau[(size_t)qi * a.n_edges + idx] = S->base_tau;
}

// Where an ant stands after stepping back to position `len` of its route (len > 0: the head of road
// route[len - 1]; len = 0: src): the node, its CSR row and its remaining bound h. Every lane of the
// group reads the same words; route[] was written by the group's lane 0 before a __syncwarp.
struct StandPoint {
    uint32_t u, beg, end, h;
};
__device__ __forceinline__ StandPoint stand_after_back(const ConstructArgs& a, const uint2* th, const uint32_t* route,
                                                       uint32_t len, uint32_t src, uint32_t qi) {
    StandPoint p;
    if (len == 0u) {
        p.u = src;
        p.beg = __ldg(a.row_ptr + src);
        p.end = __ldg(a.row_ptr + src + 1);
        p.h = a.qs[qi].h_src;
    } else {
        const uint32_t e = route[len - 1u];
        const uint4 r = __ldg(reinterpret_cast<const uint4*>(a.rec + e));
        const uint32_t cd = __ldg(&a.rec[e].cyc_deg);
        p.u = r.x;
        p.beg = r.y;
        p.end = r.y + (cd >> 24);
        p.h = __ldg(&th[e].y);
    }
    return p;
}

// Bits of the nodes a finished walk visited, cleared so the bitmap is clean for the next ant: the whole
// bitmap when that is cheaper, else src, the heads of the route's roads and the nodes its steps back left
// (kept at the back of the route buffer).
__device__ __forceinline__ void forget_visited(const ConstructArgs& a, uint32_t* tabu, const uint32_t* route,
                                               uint32_t src, uint32_t len, uint32_t pops, uint32_t moves,
                                               uint32_t lane, uint32_t G) {
    if (a.tabu_words <= 2u * (moves + 1u)) {
        for (uint32_t w = lane; w < a.tabu_words; w += G) tabu[w] = 0;
        return;
    }
    if (lane == 0) atomicAnd(tabu + (src >> 5), ~(1u << (src & 31)));
    for (uint32_t i = lane; i < len; i += G) {
        const uint32_t v = __ldg(a.col + route[i]);
        atomicAnd(tabu + (v >> 5), ~(1u << (v & 31)));
    }
    for (uint32_t i = lane; i < pops; i += G) {
        const uint32_t v = route[a.max_steps - 1u - i];
        atomicAnd(tabu + (v >> 5), ~(1u << (v & 31)));
    }
}

// ------------------------------------------------------------------------------------------------
// Ant construction. G lanes of a warp serve one ant (sub-warp group); lane l holds the candidates
// l, l+G, ..., l+(K-1)G of the current node's CSR row. Per step: one round of independent 16-byte
// record loads and pheromone loads, scores, a group max, integer weights, a shuffle prefix sum,
// one Philox draw, a ballot to find the chosen road and shuffles to broadcast it. At a node with no
// candidate the ant steps back to the previous node of its route (its clock and wait come back; the node
// it leaves stays visited and is noted at the back of the route buffer).
// Groups take ants from a per-iteration ticket counter, so short walks free lanes for waiting ants.
// ------------------------------------------------------------------------------------------------
template <int G, int K>
__device__ __forceinline__ void walk_ant(const ConstructArgs& a, const DevQuery& q, uint32_t qi, uint32_t k,
                                         uint32_t it, uint32_t* tabu, uint32_t lane, uint32_t gmask, uint32_t gbase) {
    constexpr int NC = G * K;              // candidate slots of the group
    constexpr bool kGather = NC <= 16;     // every lane gathers all scores and picks locally
    const uint2* __restrict__ th = a.th + (size_t)qi * a.n_edges;
    const float base_tf = a.sparse ? __uint_as_float(a.qs[qi].base_tf) : 0.0f;
    const bool frac = (q.active & kQueryFracExp) != 0u;
    const uint32_t slot = q.ant_base + k;
    uint32_t* route = a.routes + (size_t)slot * a.max_steps;
    uint32_t* rwait = a.rwait + (size_t)slot * a.max_steps;
    const uint32_t s0 = (uint32_t)q.seed, s1 = (uint32_t)(q.seed >> 32);
    uint32_t u = q.src;
    uint32_t beg = __ldg(a.row_ptr + u), end = __ldg(a.row_ptr + u + 1);
    uint32_t hu = a.qs[qi].h_src;  // remaining bound where the ant stands
    uint32_t t = 0, W = 0, steps = 0, len = 0, pops = 0, status;
    uint32_t rb_base = 0, rb_x = 0, rb_y = 0;  // lane l holds the draw of move rb_base + l
    bool rb_valid = false;
    if (lane == 0) atomicOr(tabu + (u >> 5), 1u << (u & 31));
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
        uint4 r0[K], r1[K];
        float tf[K];
        uint32_t he[K];
        uint32_t valid = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {  // slots past the row read road 0 (always in bounds) and are masked
            const uint32_t idx = lane + (uint32_t)j * G;
            const bool ok = j < nslots && idx < deg;
            valid |= (ok ? 1u : 0u) << j;
            const uint32_t e = ok ? beg + idx : 0u;
            const uint4* rp = reinterpret_cast<const uint4*>(a.rec + e);
            r0[j] = __ldg(rp);
            r1[j] = __ldg(rp + 1);
            const uint2 ph = __ldg(th + e);
            tf[j] = ph.x ? __uint_as_float(ph.x) : base_tf;  // 0: the road still holds the baseline
            he[j] = ph.y;
        }
        // 2. the draw of this move depends on (iteration, ant, move) only: the group's lanes compute the
        //    draws of the next G moves together, one each (overlapping the loads), and a move takes its
        //    draw with a shuffle
        if (!rb_valid || steps - rb_base >= (uint32_t)G) {
            const uint4 o = philox4x32_10(make_uint4(it, k, steps + lane, 0u), s0, s1);
            rb_x = o.x;
            rb_y = o.y;
            rb_base = steps;
            rb_valid = true;
        }
        const uint32_t rsrc = steps - rb_base;
        const unsigned long long rnd = (unsigned long long)__shfl_sync(gmask, rb_x, rsrc, G) |
                                       ((unsigned long long)__shfl_sync(gmask, rb_y, rsrc, G) << 32);
        // 3. candidates, waits, scores
        uint32_t cmask = 0, cong = 0;
        uint32_t sb[K], wv[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t v = r0[j].x, cy = r1[j].x & kCycleMask;
            const bool unvisited = !((tabu[v >> 5] >> (v & 31)) & 1u);
            cmask |= ((valid >> j) & (unvisited ? 1u : 0u)) << j;
            cong |= (r0[j].w >> 31) << j;
            const uint32_t sw = signal_wait(a.t_dep + t + r0[j].z, cy | (cy == 0u), r1[j].w, r1[j].y, r1[j].z);
            const uint32_t w = (v != q.dst && cy != 0u) ? sw + (r0[j].w & kQdMask) : 0u;
            wv[j] = w;
            sb[j] = __float_as_uint(score_q(tf[j], q.alpha, reduced_cost(r0[j].z + w + he[j], hu), q.beta, frac));
        }
        if (a.thr_on) {  // congested roads drop out unless every candidate is congested
            const uint32_t any_ok = __ballot_sync(gmask, (cmask & ~cong) != 0u) & gmask;
            const uint32_t any_cg = __ballot_sync(gmask, (cmask & cong) != 0u) & gmask;
            if (any_ok && any_cg) cmask &= ~cong;
        }
        if ((__ballot_sync(gmask, cmask != 0u) & gmask) == 0u) {
            if (len == 0) {  // back at src with no road left
                status = kAntDeadEnd;
                break;
            }
            // step back: leave u (it stays visited), return to the tail of route[len - 1] with its clock
            if (lane == 0) route[a.max_steps - 1u - pops] = u;
            ++pops;
            --len;
            const uint32_t e_in = route[len], w_in = rwait[len];
            t -= __ldg(&a.rec[e_in].tt) + w_in;
            W -= w_in;
            const StandPoint p = stand_after_back(a, th, route, len, q.src, qi);
            u = p.u;
            beg = p.beg;
            end = p.end;
            hu = p.h;
            ++steps;
            __syncwarp(gmask);
            continue;
        }
        int pick_lane, pick_slot;
        if constexpr (kGather) {
            // 4. largest candidate score of the group (non-negative floats order like their bits)
            uint32_t mb = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) mb = max(mb, (cmask >> j & 1u) ? sb[j] : 0u);
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(gmask, mb, off, G));
            // 5. own integer weights; every lane gathers the group's weights and picks locally
            const WeightScale sc = weight_scale(mb);
            uint32_t incl[NC];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const uint32_t mine = (cmask >> j & 1u) ? roulette_weight_f(sb[j], sc) : 0u;
#pragma unroll
                for (int l = 0; l < G; ++l) incl[j * G + l] = j < nslots ? __shfl_sync(gmask, mine, l, G) : 0u;
            }
#pragma unroll
            for (int h = 1; h < NC; h <<= 1)  // inclusive running sums in log depth (Kogge-Stone)
#pragma unroll
                for (int i = NC - 1; i >= h; --i) incl[i] += incl[i - h];
            // roulette: the first candidate (CSR order = index lane + j*G) whose running weight exceeds
            // r is the number of running weights <= r
            const uint32_t r = draw_index(rnd, incl[NC - 1]);
            int pick = 0;
#pragma unroll
            for (int i = 0; i < NC; ++i) pick += incl[i] <= r ? 1 : 0;
            pick_lane = pick % G;
            pick_slot = pick / G;
        } else {
            // 4. largest score of the group (non-negative floats order like their bit patterns)
            uint32_t mb = 0;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if ((cmask >> j & 1u) && sb[j] > mb) mb = sb[j];
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(gmask, mb, off, G));
            // 5. integer weights, inclusive prefix in CSR order (index lane + j*G) by shuffles, roulette
            const WeightScale sc = weight_scale(mb);
            uint32_t carry = 0, incl[K];
            uint32_t wt[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                wt[j] = 0;
                incl[j] = carry;
                if (j < nslots) {
                    wt[j] = (cmask >> j & 1u) ? roulette_weight_f(sb[j], sc) : 0u;
                    uint32_t xs = wt[j];
#pragma unroll
                    for (int d = 1; d < G; d <<= 1) {
                        const uint32_t y = __shfl_up_sync(gmask, xs, d, G);
                        if (lane >= (uint32_t)d) xs += y;
                    }
                    incl[j] = carry + xs;
                    carry = __shfl_sync(gmask, incl[j], G - 1, G);
                }
            }
            const uint32_t r = draw_index(rnd, carry);
            int js = -1;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (wt[j] != 0u && incl[j] - wt[j] <= r && r < incl[j]) js = j;
            const uint32_t bw = __ballot_sync(gmask, js >= 0) & gmask;
            pick_lane = (__ffs(bw) - 1) - (int)gbase;
            pick_slot = __shfl_sync(gmask, js, pick_lane, G);
        }
        // 6. the chosen candidate's data from the lane that evaluated it
        uint32_t c_h = 0, c_vb = 0, c_ve = 0, c_tt = 0, c_w = 0, c_he = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (pick_slot == j) {
                c_h = r0[j].x;
                c_vb = r0[j].y;
                c_ve = r0[j].y + (r1[j].x >> 24);
                c_tt = r0[j].z;
                c_w = wv[j];
                c_he = he[j];
            }
        c_h = __shfl_sync(gmask, c_h, pick_lane, G);
        c_vb = __shfl_sync(gmask, c_vb, pick_lane, G);
        c_ve = __shfl_sync(gmask, c_ve, pick_lane, G);
        c_tt = __shfl_sync(gmask, c_tt, pick_lane, G);
        c_w = __shfl_sync(gmask, c_w, pick_lane, G);
        c_he = __shfl_sync(gmask, c_he, pick_lane, G);
        // 7. position update
        const uint32_t e = beg + (uint32_t)pick_lane + (uint32_t)pick_slot * G;
        t += c_tt + c_w;
        W += c_w;
        u = c_h;
        beg = c_vb;
        end = c_ve;
        hu = c_he;
        if (lane == 0) {
            route[len] = e;
            rwait[len] = c_w;
            atomicOr(tabu + (u >> 5), 1u << (u & 31));
        }
        ++len;
        ++steps;
        __syncwarp(gmask);
        if (t > kTCap) {
            status = kAntTimeCap;
            break;
        }
    }
    QueryState* S = a.qs + qi;
    if (lane == 0) {
        a.ant_steps[slot] = len;
        a.ant_wait[slot] = W;
        atomicAdd(&S->steps, (unsigned long long)steps);
        if (status == kAntSuccess) atomicAdd(&S->nsucc, 1ull);
        if (a.ant_log) {
            uint32_t* l = a.ant_log + 4ull * (q.log_base + (uint64_t)it * q.n_ants + k);
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
        if (lane == 0) atomicMin(&S->best_key, ((unsigned long long)t << 32) | ((unsigned long long)it * q.n_ants + k));
    }
    forget_visited(a, tabu, route, q.src, len, pops, steps, lane, G);
    __syncwarp(gmask);
}

}  // namespace gmp

// Device routines shared by the iteration kernels (gmp_kernels.cu) and the persistent job
// (gmp_persistent.cu): the sub-warp ant walk and the preemptive phase order of one intersection.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp_device.cuh"
#include "gmp_internal.h"

namespace gmp {

// ------------------------------------------------------------------------------------------------
// Queue / preemption update of one intersection (Calc_Dens / Comp_Thres; Fig. 3 signal block).
// Queues and storage per phase come from the intersection's approaches; the phase order is (1) phases
// whose queue exceeds 3/4 of their storage, longest first; else (2) phases red for longer than a cycle,
// longest first; else (3) the longest non-empty queue; then the remaining non-empty phases, then the
// empty ones, each in index order. Every approach's record then gets its green window under that order.
//
// FULL passes (densities, red times or signals changed) rewrite each approach's whole 32-byte record,
// so no record is left half written; TICK passes first apply the tick's discharge to the vehicles. The
// other passes (the per-iteration update within a job, where densities and red times are fixed)
// recompute the order and rewrite an intersection's order and green windows only where the order
// differs from the stored one: the records are a function of the order and of the fixed tables.
// ------------------------------------------------------------------------------------------------

// Vehicles on the road of approach slot i. In a tick pass the road first loses what it discharged
// (leave) and gains its share of its tail's discharge K: K / d each for the tail's d out-roads and one
// more for the first K mod d of them in CSR order. The new count is stored (modulo 2^32, like the word).
template <bool TICK>
__device__ __forceinline__ uint32_t approach_vehicles(const QueueTables& t, uint32_t i) {
    if (!TICK) return t.veh[i];
    const uint32_t u = t.in_tail[i], e = t.in_edge[i];
    const uint32_t rb = t.row_ptr[u], d = t.row_ptr[u + 1] - rb;  // d >= 1: road e leaves u
    const unsigned long long k = t.K[u];
    uint32_t share, extra;
    if ((k >> 32) == 0) {
        share = (uint32_t)k / d;
        extra = (uint32_t)k - share * d;
    } else {
        const unsigned long long q = k / d;
        share = (uint32_t)q;
        extra = (uint32_t)(k - q * d);
    }
    const uint32_t n = t.veh[i] - t.leave[i] + share + (e - rb < extra ? 1u : 0u);
    t.veh[i] = n;
    return n;
}

// First half of a road's record (see EdgeRec) for a road into v carrying n vehicles, with jam capacity
// c, free-flow time ff and `lanes` lanes: the head, its CSR row, the congested travel time, the queue
// delay at a signalised head and the congestion flag.
__device__ __forceinline__ uint4 road_front(const QueueTables& t, uint32_t v, uint32_t vbeg, bool signalised,
                                            uint32_t n, uint32_t c, uint32_t ff, uint32_t lanes) {
    uint32_t qd = 0;
    if (signalised) {
        const uint64_t d = mul_div_u32(n, t.h_sat, lanes);
        qd = d > kTimeClamp ? kTimeClamp : (uint32_t)d;
    }
    const uint32_t fl = (t.thr != kThrOff && (uint64_t)n * 1000u > (uint64_t)t.thr * c) ? 1u : 0u;
    return make_uint4(v, vbeg, edge_time_ms(ff, c, n), qd | (fl << 31));
}

// The same for approach slot i, from the slot tables.
__device__ __forceinline__ uint4 record_front(const QueueTables& t, uint32_t i, uint32_t v, uint32_t vbeg,
                                              bool signalised, uint32_t n) {
    return road_front(t, v, vbeg, signalised, n, t.cap[i], t.ff[i], t.lanes[i]);
}

constexpr uint32_t kOrderId0 = 0x03020100u, kOrderId1 = 0x07060504u;  // identity order, 4 phases a word

// An unsignalised intersection: identity order, no wait, and its out-degree in every approach's record.
template <bool FULL, bool TICK>
__device__ __forceinline__ void queue_unsignalised(const QueueTables& t, uint32_t v, uint32_t vb, uint32_t deg,
                                                   uint32_t ib, uint32_t ie, uint2* ord) {
    if (!FULL) {
        const uint2 o = *ord;
        if (o.x == kOrderId0 && o.y == kOrderId1) return;
    }
    *ord = make_uint2(kOrderId0, kOrderId1);
    for (uint32_t i = ib; i < ie; ++i) {
        uint4* r = reinterpret_cast<uint4*>(t.rec + t.in_edge[i]);
        if (FULL) r[0] = record_front(t, i, v, vb, false, approach_vehicles<TICK>(t, i));
        r[1] = make_uint4(deg, 0u, 0u, 0u);
    }
}

// Any intersection (up to 8 phases). Phase-indexed values stay in registers: they are read and written
// at compile-time indices only (loops over the 8 possible phases are unrolled and masked).
template <bool FULL, bool TICK>
__device__ __forceinline__ void queue_node(uint32_t v, const QueueTables& t) {
    static_assert(FULL || !TICK, "a tick pass rewrites whole records");
    const uint32_t N = t.n_nodes, P = t.nph[v], ib = t.in_ptr[v], ie = t.in_ptr[v + 1];
    const uint32_t vb = t.row_ptr[v];
    const uint32_t deg = min(t.row_ptr[v + 1] - vb, 255u) << 24;  // out-degree of v (at most 128 runs)
    uint2* const ord = reinterpret_cast<uint2*>(t.order + (size_t)v * kMaxPhases);
    if (P == 0) {
        queue_unsignalised<FULL, TICK>(t, v, vb, deg, ib, ie, ord);
        return;
    }
    uint64_t Q[kMaxPhases], S[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) Q[k] = S[k] = 0;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t n = approach_vehicles<TICK>(t, i);
        const uint32_t p = t.ephase[i] & (kMaxPhases - 1), c = t.cap[i];
#pragma unroll
        for (uint32_t k = 0; k < kMaxPhases; ++k) {
            Q[k] += p == k ? n : 0u;
            S[k] += p == k ? c : 0u;
        }
    }
    const uint32_t cy = t.cycle[v];
    uint32_t over = 0, starved = 0, nonempty = 0;
    uint32_t rd[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        rd[k] = k < P ? t.red[(size_t)k * N + v] : 0u;
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
    // the empty ones, each in index order; a phase's position in the plan is its rank by key, and the
    // phases at or above P keep their own positions
    constexpr uint64_t kVmax = (1ull << 48) - 1;
    uint64_t key[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        const uint64_t val = by_q ? Q[k] : (uint64_t)rd[k];
        const uint64_t grp = (prio >> k & 1u) ? 0u : ((nonempty >> k & 1u) ? 1u : 2u);
        key[k] = (grp << 60) | (grp == 0 ? (kVmax - (val < kVmax ? val : kVmax)) << 4 : 0u) | k;
    }
    uint32_t before[kMaxPhases];  // per phase: the phases ahead of it in the plan
    uint32_t lo = 0, hi = 0;      // the plan, one byte per position
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        uint32_t rank = 0, bm = 0;
#pragma unroll
        for (uint32_t q = 0; q < kMaxPhases; ++q)
            if (q < P && key[q] < key[k]) {
                ++rank;
                bm |= 1u << q;
            }
        before[k] = bm;
        const uint32_t pos = k < P ? rank : k;
        if (pos < 4u) lo |= k << (8u * pos);
        else hi |= k << (8u * (pos - 4u));
    }
    if (!FULL) {
        const uint2 o = *ord;
        if (o.x == lo && o.y == hi) return;
    }
    *ord = make_uint2(lo, hi);
    uint32_t gr[kMaxPhases], start[kMaxPhases];
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) gr[k] = k < P ? t.green[(size_t)k * N + v] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kMaxPhases; ++k) {
        uint32_t st = 0;
#pragma unroll
        for (uint32_t q = 0; q < kMaxPhases; ++q) st += (before[k] >> q & 1u) ? gr[q] : 0u;
        start[k] = st;
    }
    const uint32_t off = t.offset[v];
    const uint32_t magic = 0xFFFFFFFFu / cy;
    for (uint32_t i = ib; i < ie; ++i) {
        const uint32_t p = t.ephase[i] & (kMaxPhases - 1);
        uint32_t st = 0, gl = 0;
#pragma unroll
        for (uint32_t k = 0; k < kMaxPhases; ++k) {
            st = p == k ? start[k] : st;
            gl = p == k ? gr[k] : gl;
        }
        uint4* r = reinterpret_cast<uint4*>(t.rec + t.in_edge[i]);
        if (FULL) r[0] = record_front(t, i, v, vb, true, t.veh[i]);
        r[1] = make_uint4(cy | deg, (off + st) % cy, gl, magic);
    }
}

// Up to four approach slots of one intersection, in registers.
struct ApproachBatch {
    uint32_t n[4], cap[4], ph[4];  // vehicles, jam capacity, approach phase
    uint32_t e[4], ff[4], ln[4];   // road id, free-flow time, lanes (whole-record passes only)
};

// Load slots [i0, i0 + cnt), cnt <= 4, issuing every load of the batch before any is used. In a tick pass
// the discharge is then applied and the new vehicle counts are stored (as approach_vehicles does).
template <bool FULL, bool TICK>
__device__ __forceinline__ void load_batch(const QueueTables& t, uint32_t i0, uint32_t cnt, ApproachBatch& b) {
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        const bool ok = j < cnt;
        const uint32_t i = i0 + j;
        b.n[j] = ok ? t.veh[i] : 0u;
        b.cap[j] = ok ? t.cap[i] : 0u;
        b.ph[j] = ok ? t.ephase[i] : 0u;
        b.e[j] = (FULL && ok) ? t.in_edge[i] : 0u;
        b.ff[j] = (FULL && ok) ? t.ff[i] : 0u;
        b.ln[j] = (FULL && ok) ? t.lanes[i] : 1u;
    }
    if (TICK) {
        uint32_t u[4], lv[4], rb[4], re[4];
        unsigned long long k[4];
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const bool ok = j < cnt;
            u[j] = ok ? t.in_tail[i0 + j] : 0u;
            lv[j] = ok ? t.leave[i0 + j] : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const bool ok = j < cnt;
            rb[j] = ok ? t.row_ptr[u[j]] : 0u;
            re[j] = ok ? t.row_ptr[u[j] + 1] : 1u;
            k[j] = ok ? t.K[u[j]] : 0ull;
        }
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            if (j < cnt) {
                const uint32_t d = re[j] - rb[j];  // >= 1: the slot's road leaves u
                uint32_t share, extra;
                if ((k[j] >> 32) == 0) {
                    share = (uint32_t)k[j] / d;
                    extra = (uint32_t)k[j] - share * d;
                } else {
                    const unsigned long long q = k[j] / d;
                    share = (uint32_t)q;
                    extra = (uint32_t)(k[j] - q * d);
                }
                b.n[j] = b.n[j] - lv[j] + share + (b.e[j] - rb[j] < extra ? 1u : 0u);
                t.veh[i0 + j] = b.n[j];
            }
        }
    }
}

// Queues and storage of phases 0 and 1 from a batch.
__device__ __forceinline__ void add_batch(const ApproachBatch& b, uint32_t cnt, uint64_t& Q0, uint64_t& Q1, uint64_t& S0,
                                          uint64_t& S1) {
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        if (j < cnt) {
            const bool p1 = (b.ph[j] & (kMaxPhases - 1)) != 0u;
            Q0 += p1 ? 0u : b.n[j];
            S0 += p1 ? 0u : b.cap[j];
            Q1 += p1 ? b.n[j] : 0u;
            S1 += p1 ? b.cap[j] : 0u;
        }
    }
}

// Write the records of a batch: the whole record in FULL passes, the green window (back half) otherwise;
// back0 / back1 are the back halves of phase 0 and phase 1 approaches.
template <bool FULL>
__device__ __forceinline__ void write_batch(const QueueTables& t, uint32_t i0, uint32_t cnt, const ApproachBatch& b,
                                            uint32_t v, uint32_t vb, bool signalised, uint4 back0, uint4 back1) {
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        if (j < cnt) {
            const uint32_t e = FULL ? b.e[j] : t.in_edge[i0 + j];
            uint4* r = reinterpret_cast<uint4*>(t.rec + e);
            if (FULL) r[0] = road_front(t, v, vb, signalised, b.n[j], b.cap[j], b.ff[j], b.ln[j]);
            r[1] = (b.ph[j] & (kMaxPhases - 1)) != 0u ? back1 : back0;
        }
    }
}

// The plan of an intersection with at most two phases, as the first word of its order (the second word
// is always the identity): the rule of queue_node reduced to two sort keys, from the queues and storages
// of phases 0 and 1 and their red times. Phase 0 goes first when its key is the smaller one.
__device__ __forceinline__ uint32_t small_plan(uint32_t P, uint64_t Q0, uint64_t Q1, uint64_t S0, uint64_t S1,
                                               uint32_t rd0, uint32_t rd1, uint32_t cy) {
    if (P == 0) return kOrderId0;  // unsignalised: identity order
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
    constexpr uint64_t kVmax = (1ull << 48) - 1;
    const uint64_t v0 = by_q ? Q0 : (uint64_t)rd0, v1 = by_q ? Q1 : (uint64_t)rd1;
    const uint64_t grp0 = (prio & 1u) ? 0u : ((nonempty & 1u) ? 1u : 2u);
    const uint64_t grp1 = (prio & 2u) ? 0u : ((nonempty & 2u) ? 1u : 2u);
    const uint64_t key0 = (grp0 << 60) | (grp0 == 0 ? (kVmax - (v0 < kVmax ? v0 : kVmax)) << 4 : 0u);
    const uint64_t key1 = (grp1 << 60) | (grp1 == 0 ? (kVmax - (v1 < kVmax ? v1 : kVmax)) << 4 : 0u) | 1u;
    return (P == 1 || key0 < key1) ? kOrderId0 : 0x03020001u;
}

// queue_node for an intersection with at most two phases (unsignalised nodes, and every junction the
// generators build), with the same results in far fewer registers: two keys decide the whole order.
// Returns false, doing nothing, for an intersection with more phases (queue_node handles those). The
// phase of a road into a signalised node is below its phase count and the greens add up to the cycle
// (both checked when the signals are set), so only phases 0 and 1 occur here. The intersection's own
// words (its phase planes exist for every node) and its first four approaches are loaded up front, so
// the pass costs about two memory round trips per intersection.
template <bool FULL, bool TICK>
__device__ __forceinline__ bool queue_node_small(uint32_t v, const QueueTables& t) {
    static_assert(FULL || !TICK, "a tick pass rewrites whole records");
    const uint32_t N = t.n_nodes;
    uint2* const ord = reinterpret_cast<uint2*>(t.order + (size_t)v * kMaxPhases);
    const uint32_t P = t.nph[v], ib = t.in_ptr[v], ie = t.in_ptr[v + 1];
    const uint32_t cy = t.cycle[v];
    const uint32_t rd0 = t.red[v], rd1 = t.red[(size_t)N + v];
    const uint2 old = FULL ? make_uint2(0u, 0u) : *ord;
    uint32_t vb = 0, ve = 0, g0 = 0, g1 = 0, off = 0;
    if (FULL) {
        vb = t.row_ptr[v];
        ve = t.row_ptr[v + 1];
        g0 = t.green[v];
        g1 = t.green[(size_t)N + v];
        off = t.offset[v];
    }
    if (P > 2) return false;
    const uint32_t cnt = ie - ib, c0 = cnt < 4u ? cnt : 4u;
    ApproachBatch a;
    load_batch<FULL, TICK>(t, ib, c0, a);
    uint64_t Q0 = 0, Q1 = 0, S0 = 0, S1 = 0;
    add_batch(a, c0, Q0, Q1, S0, S1);
    for (uint32_t i0 = ib + 4; i0 < ie; i0 += 4) {  // intersections with more than four approaches
        ApproachBatch b;
        const uint32_t m = ie - i0 < 4u ? ie - i0 : 4u;
        load_batch<FULL, TICK>(t, i0, m, b);
        add_batch(b, m, Q0, Q1, S0, S1);
    }
    const uint32_t lo = small_plan(P, Q0, Q1, S0, S1, rd0, rd1, cy);
    const bool first0 = lo == kOrderId0;
    if (!FULL) {
        if (old.x == lo && old.y == kOrderId1) return true;
        vb = t.row_ptr[v];  // the order changed: what the green windows need
        ve = t.row_ptr[v + 1];
        g0 = t.green[v];
        g1 = t.green[(size_t)N + v];
        off = t.offset[v];
    }
    *ord = make_uint2(lo, kOrderId1);
    const uint32_t deg = min(ve - vb, 255u) << 24;  // out-degree of v (at most 128 runs)
    uint4 back0 = make_uint4(deg, 0u, 0u, 0u), back1 = back0;
    if (P > 0) {
        const uint32_t st0 = first0 ? 0u : g1, st1 = first0 ? g0 : 0u;  // green-window starts in plan order
        const uint32_t magic = 0xFFFFFFFFu / cy;
        back0 = make_uint4(cy | deg, (off + st0) % cy, g0, magic);
        back1 = make_uint4(cy | deg, (off + st1) % cy, g1, magic);
    }
    write_batch<FULL>(t, ib, c0, a, v, vb, P > 0, back0, back1);
    for (uint32_t i0 = ib + 4; i0 < ie; i0 += 4) {
        ApproachBatch b;
        const uint32_t m = ie - i0 < 4u ? ie - i0 : 4u;
        load_batch<FULL, false>(t, i0, m, b);  // vehicles as the first round left them
        write_batch<FULL>(t, i0, m, b, v, vb, P > 0, back0, back1);
    }
    return true;
}

// Marks node v visited in the bitmap of a walk whose lanes all call this with the same v: every lane
// reads the word and writes it back with the bit set, so the lanes write one value to one address, and
// whichever order their reads and writes take, the word ends with the bit set and every other bit as it
// was (no other walk writes this bitmap; the group's next reads follow a __syncwarp).
// Measured against an atomicOr by every lane (same-address atomics serialise): groups of four lanes in
// lockstep with bitmaps in global memory, 64 colonies of the 100k-node graph x 20 iterations, 106 ->
// 91 ms; the pipelined walk, 2 % less. Groups that do not step in lockstep keep the atomic: with bitmaps in global memory
// the read ahead of the write stalls each group on its own (twice the time measured).
__device__ __forceinline__ void mark_visited(uint32_t* tabu, uint32_t v) {
    const uint32_t w = v >> 5;
    tabu[w] = tabu[w] | (1u << (v & 31));
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
// group reads the same words, which every lane of the group wrote itself.
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
template <int G, int K, bool HANDOFF, bool SMEM_TABU>
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
        if (HANDOFF && a.handoff_moves && steps == a.handoff_moves) {  // a long walk: the tail kernel finishes it
            if (lane == 0) {
                const uint32_t idx = atomicAdd(a.tail_count + it, 1u);
                a.tail_list[a.ticket_base + idx] = slot;
                WalkState ws;
                ws.u = u;
                ws.beg = beg;
                ws.end = end;
                ws.hu = hu;
                ws.t = t;
                ws.W = W;
                ws.steps = steps;
                ws.len = len;
                ws.pops = pops;
                ws.qi = qi;
                ws.k = k;
                ws.pad = 0;
                a.tail_state[slot] = ws;
            }
            uint32_t* out = a.tail_tabu + (size_t)slot * a.tabu_words;
            for (uint32_t w = lane; w < a.tabu_words; w += G) out[w] = tabu[w];
            __syncwarp(gmask);  // the copy is complete before the bits are cleared for the group's next ant
            forget_visited(a, tabu, route, q.src, len, pops, steps, lane, G);
            __syncwarp(gmask);
            return;
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
            route[a.max_steps - 1u - pops] = u;  // every lane, the same word
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
        // every lane of the group writes the same words: no lane-dependent branch on the move's path
        // (measured faster than a store by one lane, for bitmaps in shared and in global memory alike)
        route[len] = e;
        rwait[len] = c_w;
        if constexpr (SMEM_TABU) mark_visited(tabu, u);  // a bitmap in global memory keeps the atomic
        else atomicOr(tabu + (u >> 5), 1u << (u & 31));
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

// ------------------------------------------------------------------------------------------------
// Pipelined walk, one ant per warp in four sub-groups of eight lanes. While the roulette of move k runs
// on the scores of the node the ant stands on (held by sub-group g, lane 8g + l for road l of the
// row), sub-group j evaluates the row of candidate j as if the ant had moved there: its loads, visited
// checks, waits and scores, at the clock and bound the ant would have there. Move k then takes sub-group
// p's evaluation as the next current row, so a move's dependent chain is the longer of the two halves
// instead of their sum. A pick beyond the fourth candidate, a step back and the start evaluate the
// stand point's row directly. The arithmetic, its inputs and the draws are walk_ant's, so the walks are
// the same. It continues a walk that walk_ant suspended (its state, route buffer and visited set), on a
// graph whose nodes have at most eight out-roads; the visited set is in the caller's shared memory.
// ------------------------------------------------------------------------------------------------
struct RowEval {  // one lane's road of a row: the fields a move needs and its score
    uint32_t head, vbeg, vend, tt, w, he, sb;
    bool ok;  // a road of the row, to an unvisited node
    bool cg;  // over the congestion threshold
};

struct RowLoad {  // the loads of one lane's road of a row
    uint4 r0, r1;
    uint2 ph;
    bool in;
};

__device__ __forceinline__ RowLoad load_road(const ConstructArgs& a, const uint2* th, uint32_t vbeg, uint32_t deg,
                                             uint32_t l) {
    RowLoad x;
    x.in = l < deg;
    const uint32_t e = x.in ? vbeg + l : 0u;  // past the row: road 0 (always in bounds), masked
    const uint4* rp = reinterpret_cast<const uint4*>(a.rec + e);
    x.r0 = __ldg(rp);
    x.r1 = __ldg(rp + 1);
    x.ph = __ldg(th + e);
    return x;
}

__device__ __forceinline__ RowEval finish_road(const ConstructArgs& a, const DevQuery& q, float base_tf, bool frac,
                                               const uint32_t* tabu, const RowLoad& ld, uint32_t t_at,
                                               uint32_t h_at) {
    const uint4 r0 = ld.r0, r1 = ld.r1;
    const uint2 ph = ld.ph;
    const float tf = ph.x ? __uint_as_float(ph.x) : base_tf;
    RowEval x;
    x.head = r0.x;
    x.vbeg = r0.y;
    x.vend = r0.y + (r1.x >> 24);
    x.tt = r0.z;
    x.he = ph.y;
    const uint32_t cy = r1.x & kCycleMask;
    x.ok = ld.in && !((tabu[x.head >> 5] >> (x.head & 31)) & 1u);
    x.cg = (r0.w >> 31) != 0u;
    const uint32_t sw = signal_wait(a.t_dep + t_at + r0.z, cy | (cy == 0u), r1.w, r1.y, r1.z);
    x.w = (x.head != q.dst && cy != 0u) ? sw + (r0.w & kQdMask) : 0u;
    x.sb = __float_as_uint(score_q(tf, q.alpha, reduced_cost(r0.z + x.w + x.he, h_at), q.beta, frac));
    return x;
}

__device__ __forceinline__ RowEval eval_road(const ConstructArgs& a, const DevQuery& q, const uint2* th,
                                             float base_tf, bool frac, const uint32_t* tabu, uint32_t vbeg,
                                             uint32_t deg, uint32_t l, uint32_t t_at, uint32_t h_at) {
    const bool in = l < deg;
    const uint32_t e = in ? vbeg + l : 0u;  // past the row: road 0 (always in bounds), masked
    const uint4* rp = reinterpret_cast<const uint4*>(a.rec + e);
    const uint4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
    const uint2 ph = __ldg(th + e);
    const float tf = ph.x ? __uint_as_float(ph.x) : base_tf;
    RowEval x;
    x.head = r0.x;
    x.vbeg = r0.y;
    x.vend = r0.y + (r1.x >> 24);
    x.tt = r0.z;
    x.he = ph.y;
    const uint32_t cy = r1.x & kCycleMask;
    x.ok = in && !((tabu[x.head >> 5] >> (x.head & 31)) & 1u);
    x.cg = (r0.w >> 31) != 0u;
    const uint32_t sw = signal_wait(a.t_dep + t_at + r0.z, cy | (cy == 0u), r1.w, r1.y, r1.z);
    x.w = (x.head != q.dst && cy != 0u) ? sw + (r0.w & kQdMask) : 0u;
    x.sb = __float_as_uint(score_q(tf, q.alpha, reduced_cost(r0.z + x.w + x.he, h_at), q.beta, frac));
    return x;
}

__device__ __forceinline__ void walk_ant_spec(const ConstructArgs& a, const DevQuery& q, uint32_t qi, uint32_t k,
                                              uint32_t it, uint32_t* tabu, uint32_t lane, const WalkState& ws) {
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t sg = lane >> 3, sl = lane & 7u;  // sub-group, lane in it
    const uint2* __restrict__ th = a.th + (size_t)qi * a.n_edges;
    const float base_tf = a.sparse ? __uint_as_float(a.qs[qi].base_tf) : 0.0f;
    const bool frac = (q.active & kQueryFracExp) != 0u;
    const uint32_t slot = q.ant_base + k;
    uint32_t* route = a.routes + (size_t)slot * a.max_steps;
    uint32_t* rwait = a.rwait + (size_t)slot * a.max_steps;
    const uint32_t s0 = (uint32_t)q.seed, s1 = (uint32_t)(q.seed >> 32);
    uint32_t u = ws.u, beg = ws.beg, end = ws.end, hu = ws.hu;  // where the suspended walk stands
    uint32_t t = ws.t, W = ws.W, steps = ws.steps, len = ws.len, pops = ws.pops, status;
    uint32_t rb_base = 0, rb_x = 0, rb_y = 0;  // lane l holds the draw of move rb_base + l
    bool rb_valid = false;
    uint32_t g = 0;  // the sub-group holding the current row
    RowEval cur = eval_road(a, q, th, base_tf, frac, tabu, beg, end - beg, sl, t, hu);
    for (;;) {
        if (u == q.dst) {
            status = kAntSuccess;
            break;
        }
        if (steps == a.max_steps) {
            status = kAntStepCap;
            break;
        }
        const uint32_t gshift = 8u * g;
        bool cand = cur.ok;
        if (a.thr_on) {  // congested roads drop out unless every candidate is congested
            const uint32_t okb = (__ballot_sync(FULL, cur.ok && !cur.cg) >> gshift) & 0xFFu;
            const uint32_t cgb = (__ballot_sync(FULL, cur.ok && cur.cg) >> gshift) & 0xFFu;
            if (okb && cgb) cand = cur.ok && !cur.cg;
        }
        if (((__ballot_sync(FULL, cand) >> gshift) & 0xFFu) == 0u) {
            if (len == 0) {  // back at src with no road left
                status = kAntDeadEnd;
                break;
            }
            route[a.max_steps - 1u - pops] = u;
            ++pops;
            --len;
            const uint32_t e_in = route[len], w_in = rwait[len];
            t -= __ldg(&a.rec[e_in].tt) + w_in;
            W -= w_in;
            const StandPoint sp = stand_after_back(a, th, route, len, q.src, qi);
            u = sp.u;
            beg = sp.beg;
            end = sp.end;
            hu = sp.h;
            ++steps;
            __syncwarp();
            cur = eval_road(a, q, th, base_tf, frac, tabu, beg, end - beg, sl, t, hu);
            g = 0;
            continue;
        }
        if (!rb_valid || steps - rb_base >= 32u) {
            const uint4 o = philox4x32_10(make_uint4(it, k, steps + lane, 0u), s0, s1);
            rb_x = o.x;
            rb_y = o.y;
            rb_base = steps;
            rb_valid = true;
        }
        const uint32_t rsrc = steps - rb_base;
        const unsigned long long rnd = (unsigned long long)__shfl_sync(FULL, rb_x, rsrc) |
                                       ((unsigned long long)__shfl_sync(FULL, rb_y, rsrc) << 32);
        // speculation: sub-group j evaluates the row of candidate j of the current row
        const uint32_t src = gshift + sg;
        const uint32_t s_vbeg = __shfl_sync(FULL, cur.vbeg, src);
        const uint32_t s_vend = __shfl_sync(FULL, cur.vend, src);
        const uint32_t s_tt = __shfl_sync(FULL, cur.tt, src);
        const uint32_t s_w = __shfl_sync(FULL, cur.w, src);
        const uint32_t s_he = __shfl_sync(FULL, cur.he, src);
        const RowLoad sld = load_road(a, th, s_vbeg, s_vend - s_vbeg, sl);
        // roulette on the current row, in every sub-group (sub-group g's is the move's)
        uint32_t mb = cand ? cur.sb : 0u;
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(FULL, mb, off, 8));
        const WeightScale sc = weight_scale(mb);
        const uint32_t mine = cand ? roulette_weight_f(cur.sb, sc) : 0u;
        const RowEval spec = finish_road(a, q, base_tf, frac, tabu, sld, t + s_tt + s_w, s_he);
        uint32_t incl[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) incl[l] = __shfl_sync(FULL, mine, l, 8);
#pragma unroll
        for (int h = 1; h < 8; h <<= 1)
#pragma unroll
            for (int i = 7; i >= h; --i) incl[i] += incl[i - h];
        const uint32_t r = draw_index(rnd, incl[7]);
        uint32_t pick = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) pick += incl[i] <= r ? 1u : 0u;
        const uint32_t p = __shfl_sync(FULL, pick, gshift);
        const uint32_t cl = gshift + p;
        const uint32_t c_h = __shfl_sync(FULL, cur.head, cl);
        const uint32_t c_vb = __shfl_sync(FULL, cur.vbeg, cl);
        const uint32_t c_ve = __shfl_sync(FULL, cur.vend, cl);
        const uint32_t c_tt = __shfl_sync(FULL, cur.tt, cl);
        const uint32_t c_w = __shfl_sync(FULL, cur.w, cl);
        const uint32_t c_he = __shfl_sync(FULL, cur.he, cl);
        const uint32_t e = beg + p;
        t += c_tt + c_w;
        W += c_w;
        u = c_h;
        beg = c_vb;
        end = c_ve;
        hu = c_he;
        route[len] = e;
        rwait[len] = c_w;
        mark_visited(tabu, u);
        ++len;
        ++steps;
        __syncwarp();
        if (p < 4u) {  // sub-group p evaluated the new stand point's row
            cur = spec;
            g = p;
        } else {
            cur = eval_road(a, q, th, base_tf, frac, tabu, beg, end - beg, sl, t, hu);
            g = 0;
        }
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
        for (uint32_t i = lane; i < len; i += 32u) {
            atomicAdd(D + route[i], delta);
            if (a.sparse) register_road(a, qi, S, route[i]);
        }
        if (lane == 0) atomicMin(&S->best_key, ((unsigned long long)t << 32) | ((unsigned long long)it * q.n_ants + k));
    }
    forget_visited(a, tabu, route, q.src, len, pops, steps, lane, 32u);
    __syncwarp();
}

}  // namespace gmp

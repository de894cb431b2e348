// One persistent launch for a whole batch of colonies (the batched form of Algorithms 1-2).
//
// Every colony (query) moves through its iterations on its own, driven by a small state machine in
// device memory:
//   ANTS(it)  groups of G lanes claim the colony's ants of iteration `it` one at a time and walk them
//             (walk_ant: Adj_Neigh, next-node roulette, Eval_Rout, position update, deposits). The
//             group that finishes the last ant keeps the best route of the iteration and opens
//   END(it)   chunks of the iteration end: Evap_Pher + Updt_Pher over the colony's roads, plus, for
//             the first colony to reach the end of iteration `it`, the per-intersection queue /
//             preemption update (Calc_Dens, Comp_Thres) over all nodes. The group that finishes the
//             last chunk moves the colony to ANTS(it + 1) or marks it finished.
// A colony never waits for another, so the job takes as long as its slowest colony rather than the
// sum over iterations of the slowest ant of any colony. Groups that find nothing to claim poll with a
// bound; when the bound expires the kernel raises an error flag and returns (GMP_ERR_TIMEOUT).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp_device.cuh"
#include "gmp_internal.h"
#include "gmp_walk.cuh"

namespace gmp {

enum : uint32_t { kPhaseAnts = 0, kPhaseEnd = 1, kPhaseDone = 2 };
constexpr uint32_t kEdgeChunk = 64;   // roads per evaporation chunk (a few per lane, all loads in flight)

__device__ __forceinline__ uint32_t load_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void k_persistent_init(uint32_t Q, uint32_t maxI, const DevQuery* __restrict__ q,
                                  IterCounters* __restrict__ ctr, uint32_t* __restrict__ qstate,
                                  uint32_t* __restrict__ qflag, uint32_t* __restrict__ misc) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = Q * maxI;
    for (uint32_t j = i; j < n; j += gridDim.x * blockDim.x) ctr[j] = IterCounters{};
    for (uint32_t j = i; j < maxI; j += gridDim.x * blockDim.x) qflag[j] = 0;
    for (uint32_t j = i; j < Q; j += gridDim.x * blockDim.x)
        qstate[j] = q[j].active ? ((0u << 2) | kPhaseAnts) : kPhaseDone;
    if (i == 0) {
        uint32_t inactive = 0;
        for (uint32_t j = 0; j < Q; ++j) inactive += q[j].active ? 0u : 1u;
        misc[0] = inactive;  // finished colonies
        misc[1] = 0;         // error flag
    }
}

template <int G, int K, bool SMEM>
__global__ void __launch_bounds__(128) k_persistent(PersistentArgs p) {
    extern __shared__ uint32_t smem[];
    const ConstructArgs& a = p.c;
    const uint32_t lane = threadIdx.x & (G - 1);
    const uint32_t gib = threadIdx.x / G;
    const uint32_t gbase = (threadIdx.x & 31u) & ~(uint32_t)(G - 1);
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << gbase);
    const uint32_t groups = blockDim.x / G;
    uint32_t* tabu = SMEM ? smem + (size_t)gib * a.tabu_words
                          : a.tabu_global + ((size_t)blockIdx.x * groups + gib) * a.tabu_words;
    if (SMEM)  // global bitmaps are cleared once per job; every walk clears its own bits when it ends
        for (uint32_t w = lane; w < a.tabu_words; w += G) tabu[w] = 0;
    __syncwarp(gmask);
    const uint32_t Q = a.n_queries, E = a.n_edges;
    const uint32_t n_edge_chunks = (E + kEdgeChunk - 1) / kEdgeChunk;
    const uint32_t node_chunk = p.node_chunk;  // intersections per queue-update chunk
    const uint32_t n_node_chunks = (p.n_nodes + node_chunk - 1) / node_chunk;
    // colony qi is served by the blocks b == qi (mod Q), so the groups of a warp share a colony and go
    // through its phases together; j is this group's rank among the colony's groups
    const uint32_t qi = blockIdx.x % Q, j = (blockIdx.x / Q) * groups + gib;
    const uint32_t ng = ((gridDim.x - qi - 1u) / Q + 1u) * groups;  // groups serving colony qi
    const DevQuery q = a.queries[qi];
    uint32_t seen = 0xFFFFFFFFu;  // last state this group worked on
    uint32_t idle = 0, nap = 32;
    for (;;) {
        // poll this colony's state word only (relaxed); the error word every 64 polls
        uint32_t st = 0, err = 0;
        if (lane == 0) {
            st = *(volatile const uint32_t*)(p.qstate + qi);
            if ((idle & 63u) == 63u) err = *(volatile const uint32_t*)(p.misc + 1);
        }
        st = __shfl_sync(gmask, st, 0, G);
        err = __shfl_sync(gmask, err, 0, G);
        if (err) break;
        const uint32_t phase = st & 3u, it = st >> 2;
        if (phase == kPhaseDone) break;
        if (st == seen) {  // this group's share of the phase is done: wait for the colony to move on
            if (++idle > p.spin_limit) {
                if (lane == 0) atomicExch(p.misc + 1, 1u);
                break;
            }
            __nanosleep(nap);
            nap = nap < 1024u ? nap * 2u : nap;
            continue;
        }
        if (lane == 0) (void)load_acquire(p.qstate + qi);  // order what follows after the state change
        __syncwarp(gmask);
        seen = st;
        idle = 0;
        nap = 32;
        IterCounters* C = p.ctr + (size_t)qi * p.max_iter + it;
        if (phase == kPhaseAnts) {
            // first ant by rank, further ants from the iteration's counter (groups that finish early
            // take the ants left over when the colony has more ants than groups)
            for (uint32_t k = j; k < q.n_ants;) {
                walk_ant<G, K, false, SMEM>(a, q, qi, k, it, tabu, lane, gmask, gbase);
                __threadfence();  // this ant's route, records and deposits before it counts as done
                __syncwarp(gmask);
                uint32_t d = 0;
                if (lane == 0) d = atomicAdd(&C->ant_done, 1u) + 1u;
                d = __shfl_sync(gmask, d, 0, G);
                if (d == q.n_ants) {  // last ant of the iteration: best route, then open the iteration end
                    __threadfence();
                    QueryState* S = a.qs + qi;
                    const unsigned long long key = S->best_key;
                    if (key != kNoKey && (uint32_t)key / q.n_ants == it) {
                        const uint32_t slot = q.ant_base + (uint32_t)key % q.n_ants;
                        const uint32_t len = a.ant_steps[slot];
                        for (uint32_t i = lane; i < len; i += G)
                            p.best_route[(size_t)qi * a.max_steps + i] = a.routes[(size_t)slot * a.max_steps + i];
                        if (lane == 0) {
                            S->best_len = len;
                            S->best_W = a.ant_wait[slot];
                        }
                    }
                    if (lane == 0) {
                        const bool owner = atomicCAS(p.qflag + it, 0u, qi + 1u) == 0u;
                        C->chunk_total = n_edge_chunks + (owner ? n_node_chunks : 0u);
                        __threadfence();
                        store_release(p.qstate + qi, (it << 2) | kPhaseEnd);
                    }
                    __syncwarp(gmask);
                }
                if (ng >= q.n_ants) break;
                uint32_t nk = 0;
                if (lane == 0) nk = ng + atomicAdd(&C->ant_claim, 1u);
                k = __shfl_sync(gmask, nk, 0, G);
            }
        } else {  // kPhaseEnd: this group's chunks of the iteration end
            uint32_t total = 0;
            if (lane == 0) total = *(volatile uint32_t*)&C->chunk_total;
            total = __shfl_sync(gmask, total, 0, G);
            for (uint32_t c = j; c < total; c += ng) {
                if (c < n_edge_chunks) {  // Evap_Pher + Updt_Pher on roads [e0, e1) of this colony
                    const uint64_t rf = q.rho_fix;
                    uint64_t* T = p.tau + (size_t)qi * E;
                    uint32_t* TF = reinterpret_cast<uint32_t*>(p.th + (size_t)qi * E);  // pheromone halves
                    unsigned long long* D = a.dep + (size_t)qi * E;
                    constexpr int PER = (int)(kEdgeChunk / G);
                    const uint32_t e0 = c * kEdgeChunk;
                    uint64_t tv[PER];
                    unsigned long long dv[PER];
#pragma unroll
                    for (int i = 0; i < PER; ++i) {  // issue every load of the chunk first
                        const uint32_t e = e0 + lane + (uint32_t)i * G;
                        tv[i] = e < E ? T[e] : 0;
                        dv[i] = e < E ? D[e] : 0;
                    }
#pragma unroll
                    for (int i = 0; i < PER; ++i) {
                        const uint32_t e = e0 + lane + (uint32_t)i * G;
                        if (e < E) {
                            const uint64_t nt = tau_next(tv[i], rf, dv[i], p.flags);
                            T[e] = nt;
                            TF[2 * (size_t)e] = tau_word(nt, p.flags);
                            D[e] = 0;
                        }
                    }
                } else {  // queue / preemption update of intersections [v0, v1) (densities fixed: same order)
                    const uint32_t v0 = (c - n_edge_chunks) * node_chunk, v1 = min(p.n_nodes, v0 + node_chunk);
                    for (uint32_t v = v0 + lane; v < v1; v += G) queue_node<false, false>(v, p.qt);
                }
                __threadfence();
                __syncwarp(gmask);
                uint32_t d = 0;
                if (lane == 0) d = atomicAdd(&C->chunk_done, 1u) + 1u;
                d = __shfl_sync(gmask, d, 0, G);
                if (d == total && lane == 0) {  // the iteration is complete
                    __threadfence();
                    if (it + 1u < q.n_iter) {
                        store_release(p.qstate + qi, ((it + 1u) << 2) | kPhaseAnts);
                    } else {
                        store_release(p.qstate + qi, kPhaseDone);
                        atomicAdd(p.misc, 1u);
                    }
                }
                __syncwarp(gmask);
            }
        }
    }
}

cudaError_t launch_persistent_init(cudaStream_t s, uint32_t Q, uint32_t maxI, const DevQuery* q, IterCounters* ctr,
                                   uint32_t* qstate, uint32_t* qflag, uint32_t* misc) {
    const uint32_t n = Q * maxI > Q ? Q * maxI : Q;
    k_persistent_init<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(Q, maxI, q, ctr, qstate, qflag,
                                                                                   misc);
    return cudaGetLastError();
}

template <int G, int K>
static cudaError_t config_p(int device, uint32_t n_nodes, KernelConfig* out) {
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
            err = cudaFuncSetAttribute(k_persistent<G, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       64 * 1024);
            if (err != cudaSuccess) return err;
        }
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<G, K, true>, block, dyn);
    } else {
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<G, K, false>, block, 0);
    }
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidValue;
    out->lanes = G;
    out->slots = K;
    out->block = block;
    out->grid = per_sm * sms;  // every block resident: a persistent launch
    out->smem = dyn;
    out->tabu_in_smem = in_smem;
    out->lockstep = false;
    return cudaSuccess;
}

cudaError_t persistent_config(int device, int lanes, uint32_t n_nodes, uint32_t max_degree, KernelConfig* out) {
    int k = 0;
    for (int kk : {1, 2, 4})
        if ((uint32_t)(lanes * kk) >= max_degree) {
            k = kk;
            break;
        }
#define GMP_PCFG(G_, K_) \
    if (lanes == G_ && k == K_) return config_p<G_, K_>(device, n_nodes, out);
    GMP_PCFG(4, 1) GMP_PCFG(4, 2) GMP_PCFG(4, 4) GMP_PCFG(8, 1) GMP_PCFG(8, 2) GMP_PCFG(8, 4)
    GMP_PCFG(16, 1) GMP_PCFG(16, 2) GMP_PCFG(16, 4) GMP_PCFG(32, 1) GMP_PCFG(32, 2) GMP_PCFG(32, 4)
#undef GMP_PCFG
    return cudaErrorInvalidValue;
}

cudaError_t launch_persistent(cudaStream_t s, const KernelConfig& kc, const PersistentArgs& p) {
#define GMP_PLAUNCH(G_, K_)                                                                    \
    if (kc.lanes == G_ && kc.slots == K_) {                                                    \
        if (kc.tabu_in_smem) k_persistent<G_, K_, true><<<kc.grid, kc.block, kc.smem, s>>>(p); \
        else k_persistent<G_, K_, false><<<kc.grid, kc.block, 0, s>>>(p);                      \
        return cudaGetLastError();                                                             \
    }
    GMP_PLAUNCH(4, 1) GMP_PLAUNCH(4, 2) GMP_PLAUNCH(4, 4) GMP_PLAUNCH(8, 1) GMP_PLAUNCH(8, 2) GMP_PLAUNCH(8, 4)
    GMP_PLAUNCH(16, 1) GMP_PLAUNCH(16, 2) GMP_PLAUNCH(16, 4) GMP_PLAUNCH(32, 1) GMP_PLAUNCH(32, 2) GMP_PLAUNCH(32, 4)
#undef GMP_PLAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace gmp

// Host-side internals shared by the C-ABI implementation and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gmacop.h"
#include "gmp_device.cuh"

namespace gmp {

// What the per-intersection passes read and write: the queue / preemption update (Calc_Dens, Comp_Thres)
// and the serving tick. Approaches are addressed by in-slot: slot i (in_ptr[v] <= i < in_ptr[v + 1]) is
// road in_edge[i] into v, and every per-approach table below is stored in slot order, so one
// intersection's approaches are contiguous. Phase tables are phase-major (entry p * n_nodes + v), so a
// warp over consecutive intersections reads one contiguous run per phase.
struct QueueTables {
    uint32_t n_nodes;
    uint32_t h_sat;                          // saturation headway per lane, ms
    uint32_t thr;                            // congestion threshold, per mille of capacity (kThrOff: off)
    const uint32_t *row_ptr, *in_ptr, *in_edge, *in_tail;
    const uint8_t* nph;                      // phases per intersection (0: unsignalised)
    const uint32_t *cycle, *offset;
    const uint32_t* green;                   // phase-major green times
    const uint8_t *ephase, *lanes;           // per slot: approach phase at the head, lanes
    const uint32_t *cap, *ff;                // per slot: jam capacity, free-flow time (ms)
    uint32_t* veh;                           // per slot: vehicles on the road (traffic state)
    uint32_t* red;                           // phase-major red-time accumulators (traffic state)
    uint8_t* order;                          // 8 per intersection: phases in plan order (traffic state)
    EdgeRec* rec;                            // per road (by road id): the records the walk reads
    const uint32_t* leave;                   // tick: vehicles each slot's road discharged
    const unsigned long long* K;             // tick: vehicles each intersection discharged
};

// A walk suspended by the construction kernel, to be finished by the tail kernel: where it stands and
// what it has done (its route, waits and popped nodes stay in the route buffer, its visited set is copied
// out beside this record).
struct __align__(16) WalkState {
    uint32_t u, beg, end, hu;  // node, its CSR row, remaining bound
    uint32_t t, W, steps, len;  // clock, waits, moves, route length
    uint32_t pops, qi, k, pad;  // steps back so far, colony (within the launch's range), ant
};

// Arguments of the construction kernel (one iteration over every ant of the batch).
struct ConstructArgs {
    const EdgeRec* rec;
    const uint32_t* row_ptr;
    const uint32_t* col;
    const DevQuery* queries;
    const uint32_t* ant_prefix;  // Q + 1 entries: first global ant of each query
    const uint64_t* tau;         // Q * E
    const uint2* th;             // Q * E pairs: pheromone as binary32 bits (tau rounded to nearest times
                                 // 2^-32) and the heuristic of the road's head towards the destination
    unsigned long long* dep;     // Q * E deposit accumulators
    QueryState* qs;
    uint32_t* routes;            // total_ants * max_steps road ids: an ant's route from the front; the
                                 // nodes its steps back left, from the back (route length + steps back
                                 // <= moves <= max_steps, so the two never meet)
    uint32_t* rwait;             // total_ants * max_steps: the wait taken at each position of the route
    uint32_t* ant_steps;         // total_ants
    uint32_t* ant_wait;          // total_ants
    uint32_t* ant_log;           // optional: 4 words per (query, iteration, ant)
    uint32_t* tickets;           // one counter per iteration
    uint32_t* tabu_global;       // per-group visited bitmaps when they do not fit in shared memory
    uint32_t n_queries, total_ants, n_edges, max_steps;
    uint32_t tabu_words, t_dep, thr_on, tabu_in_smem;
    uint32_t kappa;              // floor(360 * 2^16 / v_max)
    uint32_t ticket_base;        // job-wide index of this launch's first ant (its colonies are a
                                 // contiguous range: queries, ant_prefix and the per-colony tables
                                 // point at the range's first colony)
    // sparse pheromone layout (sparse != 0): th[e].x == 0 marks a road without a deposit so far, whose
    // pheromone is the colony's baseline; a road's first deposit registers it in the colony's list
    uint32_t sparse;
    uint32_t tflag_words;        // words per colony of the registered-road bitmap
    uint32_t* tflag;             // Q * tflag_words
    uint32_t* list_e;            // Q * E registered roads
    uint64_t* list_tau;          // Q * E their tau
    // hand-off of long walks (shared-memory visited sets only): a walk still going after handoff_moves
    // moves is suspended; the tail kernel finishes it with one ant per warp (0: off)
    uint32_t handoff_moves;
    uint32_t* tail_count;        // per iteration: walks suspended (this launch range's counters)
    uint32_t* tail_claim;        // per iteration: suspended walks taken up by the tail kernel
    uint32_t* tail_list;         // suspended walks' ant slots, from ticket_base on
    WalkState* tail_state;       // per ant slot of the job
    uint32_t* tail_tabu;         // per ant slot of the job: tabu_words of its visited set
};

// Arguments of the fused iteration-end kernel (evaporation + deposits, best route, queue update).
struct IterEndArgs {
    uint32_t n_queries, n_edges, n_nodes, it, max_steps;
    uint32_t evap_blocks;  // blocks per colony for the evaporation (set by the launcher)
    uint32_t sparse;       // sparse pheromone layout: evaporate the registered roads and the baseline
    uint32_t flags;        // GMP_FLAG_* of the context (repulsive pheromone word, unused-only evaporation)
    uint32_t* list_e;
    uint64_t* list_tau;
    const DevQuery* q;
    uint64_t* tau;
    uint2* th;
    unsigned long long* dep;
    QueryState* qs;
    const uint32_t *routes, *ant_steps, *ant_wait;
    uint32_t* best_route;
    QueueTables qt;  // the per-iteration queue update (n_nodes above says whether this launch runs it)
};

// Per-(colony, iteration) counters of the persistent job.
struct __align__(16) IterCounters {
    uint32_t ant_claim, ant_done;       // ants handed out / finished
    uint32_t chunk_claim, chunk_done;   // iteration-end chunks handed out / finished
    uint32_t chunk_total;               // chunks of this iteration end (roads, plus nodes for one colony)
    uint32_t pad[3];
};

// Arguments of the persistent job: the walk's arguments plus the colony state machine and what the
// iteration-end chunks touch.
struct PersistentArgs {
    ConstructArgs c;
    IterCounters* ctr;      // Q * max_iter
    uint32_t* qstate;       // Q: (iteration << 2) | phase
    uint32_t* qflag;        // max_iter: colony (+1) that updates the queues for that iteration index
    uint32_t* misc;         // [0] finished colonies, [1] error flag (bounded wait expired)
    uint64_t* tau;
    uint2* th;
    uint32_t* best_route;
    QueueTables qt;
    uint32_t n_nodes, max_iter, spin_limit;
    uint32_t flags;       // GMP_FLAG_* of the context
    uint32_t node_chunk;  // intersections per queue-update chunk (8..64)
};

struct KernelConfig {
    int lanes;             // lanes per ant (G); 1 = one thread per ant
    int slots;             // candidate slots per lane (K)
    int block;             // threads per block
    int grid;              // blocks
    size_t smem;           // dynamic shared memory per block
    bool tabu_in_smem;
    bool lockstep = false;  // all ants of a warp step together (k_construct_gl / k_construct_lock)
    bool frac = false;      // some colony has non-integer exponents: the lockstep kernel's instantiation
                            // with the 2^L score (the others check each colony at run time)
};

// Launchers (gmp_kernels.cu).
// Per-slot road constants (slot i is road in_edge[i]): free-flow time, jam capacity and lanes.
cudaError_t launch_edge_static(cudaStream_t s, uint32_t E, const uint32_t* in_edge, const uint32_t* len,
                               const uint16_t* speed, const uint8_t* lanes_by_road, uint32_t* ff, uint32_t* cap,
                               uint8_t* lanes);
// dst[i] = src[idx[i]] for i < n (road order into slot order), and its inverse.
cudaError_t launch_gather_u32(cudaStream_t s, uint32_t n, const uint32_t* idx, const uint32_t* src, uint32_t* dst);
cudaError_t launch_gather_u8(cudaStream_t s, uint32_t n, const uint32_t* idx, const uint8_t* src, uint8_t* dst);
// How a queue pass treats the state it finds.
enum class QueuePass {
    kRefresh,  // vehicles, red times or signals changed: every approach's whole record is rewritten
    kTick,     // kRefresh after applying the tick's discharge (leave, K) to the vehicles
    kIterate,  // within a job: recompute every order, rewrite an intersection only where it changed
};
// The queue / preemption update of every intersection (max_phases: most phases at any of them).
cudaError_t launch_queue(cudaStream_t s, const QueueTables& t, uint32_t max_phases, QueuePass pass);
// The same for the intersections with more than two phases only (the iteration end covers the rest).
cudaError_t launch_queue_general(cudaStream_t s, const QueueTables& t, QueuePass pass);
// Tick node pass: green phase at t_now, discharge of every approach (leave, K) and the red-time update of
// phases below red_planes (the others are left as they are).
cudaError_t launch_tick_node(cudaStream_t s, const QueueTables& t, uint64_t t_now, uint32_t dt,
                             uint32_t red_planes, uint32_t* leave, unsigned long long* K);
cudaError_t launch_init_batch(cudaStream_t s, uint32_t Q, uint32_t E, const DevQuery* q, const uint32_t* col,
                              const int32_t* x, const int32_t* y, uint32_t kappa, uint32_t flags, uint64_t* tau,
                              uint2* th, unsigned long long* dep, QueryState* qs, uint32_t* tickets,
                              uint32_t n_tickets, uint32_t sparse, uint32_t* tflag, uint32_t tflag_words,
                              const uint32_t* hdist, uint32_t N, bool zero_dep);
// Exact Calc_Dist (GMP_FLAG_EXACT_H) of Q colonies into hdist (Q * N), in near-far order with threshold
// step delta (ms; work only, not results); queue (Q * 4N) and stamps (Q * 2N) are scratch; err[0] is set
// if a colony ran past its level guard.
cudaError_t launch_exact_h(cudaStream_t s, uint32_t Q, uint32_t N, const DevQuery* q, const uint32_t* in_ptr,
                           const uint32_t* in_edge, const uint32_t* in_tail, const EdgeRec* rec, uint32_t delta,
                           uint32_t level_limit, uint32_t* hdist, uint32_t* queue, uint32_t* stamps, uint32_t* err);
cudaError_t launch_materialize_tau(cudaStream_t s, uint32_t E, const QueryState* qs, const uint32_t* list_e,
                                   const uint64_t* list_tau, uint64_t* out);
cudaError_t launch_construct(cudaStream_t s, const KernelConfig& kc, const ConstructArgs& a, uint32_t it);
// The walks the construction launch of iteration it suspended, finished one per warp (pipelined walk).
cudaError_t launch_construct_tail(cudaStream_t s, const KernelConfig& kc, const ConstructArgs& a, uint32_t it);
cudaError_t construct_tail_config(int device, uint32_t n_nodes, uint32_t total_ants, KernelConfig* out);
cudaError_t launch_iter_end(cudaStream_t s, const IterEndArgs& a);
cudaError_t launch_finalize(cudaStream_t s, uint32_t Q, const DevQuery* q, const QueryState* qs,
                            const uint32_t* best_route, const uint32_t* col, uint32_t max_steps, DevResult* res,
                            uint32_t* route_out);

// Persistent job (gmp_persistent.cu).
cudaError_t launch_persistent_init(cudaStream_t s, uint32_t Q, uint32_t maxI, const DevQuery* q, IterCounters* ctr,
                                   uint32_t* qstate, uint32_t* qflag, uint32_t* misc);
cudaError_t persistent_config(int device, int lanes, uint32_t n_nodes, uint32_t max_degree, KernelConfig* out);
cudaError_t launch_persistent(cudaStream_t s, const KernelConfig& kc, const PersistentArgs& p);

// Occupancy-derived configuration for a lane count and graph size.
cudaError_t construct_config(int device, int lanes, uint32_t n_nodes, uint32_t max_degree, uint32_t total_ants,
                             KernelConfig* out);
cudaError_t construct_config_lockstep(int device, int lanes, uint32_t n_nodes, uint32_t max_degree,
                                      uint32_t total_ants, bool frac, KernelConfig* out);
int construct_max_degree(int lanes);
bool construct_thread_fits(uint32_t n_nodes);

// Context internals for the host-side layers built on the C ABI (autotuner, server) (gmp_api.cu).
constexpr uint32_t kFlagNoGraphBit = 8u;      // params.flags bit: launch kernel by kernel, no graph capture
constexpr uint32_t kFlagNoLockstepBit = 16u;  // params.flags bit: free-running groups instead of lockstep
struct CtxInfo {
    int device;
    cudaStream_t stream;
    uint32_t N, E, maxdeg;
    bool has_graph;
    uint64_t budget, used;  // device memory bound (0 = none) and bytes held
};
CtxInfo ctx_info(const gmp_ctx* c);
int ctx_fail(gmp_ctx* c, int code, const char* msg);
uint32_t default_lanes(uint32_t maxdeg);  // lanes per ant when the parameters leave it open
bool lockstep_fits(int lanes, uint32_t maxdeg);  // the warp-lockstep construction kernel covers this shape
int ctx_check_query(gmp_ctx* c, const gmp_query& q);  // the checks gmp_batch_stage applies to one query
// Server support: stream-ordered allocations for a context (before it allocates anything); move a view
// of another context's traffic state onto another holder of the same road graph; the event recorded
// after the context's last launch (nullptr before any); copy one traffic state into another context's own
// (on dst's stream); the bytes the context would hold after reserving a job of n colonies.
void ctx_set_stream_alloc(gmp_ctx* c);
int ctx_rebind_state(gmp_ctx* c, gmp_ctx* holder);
cudaEvent_t ctx_done_event(const gmp_ctx* c);
bool ctx_owns_state(const gmp_ctx* c);
int ctx_copy_state(gmp_ctx* dst, const gmp_ctx* src);
uint64_t ctx_job_bytes(gmp_ctx* c, uint32_t n, uint64_t total_ants, uint32_t max_iter);

}  // namespace gmp

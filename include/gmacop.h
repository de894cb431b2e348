/*
 * gmacop.h -- C ABI of the GB300 (sm_103a) MACO-P route colony library, libgmacop.so.
 *
 * The method is GMACO-P (Jindal & Bedi, "GMACO-P: GPU assisted Preemptive MACO algorithm for enabling
 * Smart Transportation"): ants build origin-to-destination routes over a road graph by choosing the next
 * road from pheromone and a congestion/signal-aware travel-time heuristic (Sec. 4.1, Fig. 3), successful
 * ants deposit pheromone and all roads evaporate (Fig. 3; Algorithm 2), and each signalised
 * intersection reorders its phases by the preemptive rule (Fig. 3 signal block; Algorithm 2).
 * Algorithm 1 (allocate, copy in, launch, copy out, free) is the host driver this API replaces with
 * persistent device state: the graph, signals and densities stay resident between calls.
 *
 * Conventions for every entry point:
 *   - Return value: GMP_OK (0) or a GMP_ERR_* code; gmp_strerror() names it, gmp_last_error() gives the
 *     context's last detailed message.
 *   - Host pointers (const T*) are read during the call only; the library copies what it keeps. Device
 *     pointers are named d_* and must be device memory of the context's GPU.
 *   - Units: lengths and coordinates in decimetres, speeds in km/h, times in milliseconds, pheromone in
 *     unsigned Q32.32 fixed point (2^32 == 1.0).
 *   - One context is one GPU + one road graph. A context is not thread-safe: serialise calls on it.
 *   - Work is issued on the context's stream (gmp_create / gmp_set_stream). Calls that return host data
 *     synchronise that stream; *_async calls do not.
 */
#ifndef GMACOP_H
#define GMACOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMP_OK 0
#define GMP_ERR_INVALID_ARG 1 /* argument out of range or inconsistent graph/signal data */
#define GMP_ERR_NO_ROUTE 2    /* no ant reached the destination in any iteration */
#define GMP_ERR_OOM 3         /* device allocation failed or the context's memory budget is exceeded */
#define GMP_ERR_CUDA 4        /* a CUDA runtime call failed (see gmp_last_error) */
#define GMP_ERR_TIMEOUT 5     /* a bounded device-side wait or loop expired (persistent launch, exact heuristic) */
#define GMP_ERR_UNSUPPORTED 6 /* alpha/beta outside [0, 8], more than 8 phases, degree beyond the kernel limit */
#define GMP_ERR_BUFFER 7      /* caller buffer too small; the required size is reported */
#define GMP_ERR_STATE 8       /* call out of order (e.g. solve before gmp_load_graph) */

#define GMP_MAX_PHASES 8
#define GMP_THRESHOLD_OFF 0xFFFFFFFFu
#define GMP_FLAG_RANDOM_TAU 1u /* initial pheromone 0.5 + u/2^32, u = Philox(road, 0, 0, 1) word 0 */
#define GMP_FLAG_ANT_LOG 2u    /* keep a per-(iteration, ant) log {status | length << 8, moves, T, W} */
/* The paper's own MACO-P pheromone variant (Sec. 4.1 bullets, Fig. 3, Algorithm 2), one flag per part;
 * every kernel shape and both pheromone layouts honour them. */
#define GMP_FLAG_REPULSIVE 32u    /* next-node rule prefers less pheromone: scores use (1/tau)^alpha */
#define GMP_FLAG_UNIT_DEPOSIT 64u /* Ph_road++: each successful ant adds exactly 1.0 to each road used */
#define GMP_FLAG_EVAP_UNUSED 128u /* deposits first; only roads without a deposit that iteration evaporate */
#define GMP_FLAG_PAPER_LITERAL (GMP_FLAG_REPULSIVE | GMP_FLAG_UNIT_DEPOSIT | GMP_FLAG_EVAP_UNUSED)
/* Calc_Dist exactly (Algorithm 2): h(v) = the least sum of congested travel times over a path from v to
 * the colony's destination (2^28 when there is none), computed on the GPU per colony at the start of each
 * job, in place of the straight-line bound; it also sets the deposit numerator h(src). Needs
 * Q * 28 N bytes more workspace; gmp_solve_static refuses it (GMP_ERR_UNSUPPORTED). */
#define GMP_FLAG_EXACT_H 256u

#define GMP_MODE_AUTO 0u       /* library picks */
#define GMP_MODE_ITERATIVE 1u  /* one kernel sequence per iteration, whole batch, CUDA-graph replay */
#define GMP_MODE_PERSISTENT 2u /* one persistent launch working through (query, iteration) items */

typedef struct gmp_ctx gmp_ctx;

/* Tunables of the colony (Fig. 3 leaves all of them unstated). Zero means "default" where noted. */
typedef struct {
    uint32_t max_steps;     /* moves per ant (forward or back) before it gives up; 0 = min(2(N-1), 4096),
                               enough for a complete depth-first walk; at most 2^24 */
    uint32_t h_sat_ms;      /* saturation headway per lane for queue delays; 0 = 2000 ms */
    uint32_t thr_permille;  /* Fig. 3 congestion threshold: a road with vehicles*1000 > thr*capacity is
                               avoided unless every candidate is; GMP_THRESHOLD_OFF disables it */
    uint32_t flags;         /* GMP_FLAG_* */
    uint32_t t_dep_ms;      /* departure clock for signal phases, < 2^30 */
    uint32_t lanes_per_ant; /* lanes of a warp that evaluate one ant's candidates: 0 (autotune), 4, 8, 16, 32 */
    uint32_t mode;          /* GMP_MODE_* */
    uint32_t queue_chunk;   /* persistent mode: intersections per queue-update work item; 0 (= 16), 8, 16,
                               32 or 64 */
    uint32_t branches;      /* iterative mode: the colonies are split into this many contiguous ranges that
                               run as concurrent chains of launches; 0 = min(colonies, 16), at most 64 */
    uint32_t tau_layout;    /* pheromone tables: GMP_TAU_AUTO, GMP_TAU_DENSE or GMP_TAU_SPARSE (same results) */
    uint32_t poll_limit;    /* persistent mode: polls a group waiting for its colony's next phase makes before
                               the job stops and reports GMP_ERR_TIMEOUT; 0 = 2^23 (seconds) */
    uint32_t level_limit;   /* GMP_FLAG_EXACT_H: relaxation levels before the heuristic's pass stops and the
                               job reports GMP_ERR_TIMEOUT; 0 = 4N + 4096 */
    uint32_t handoff_moves; /* iterative mode with sub-warp groups that do not step in lockstep, on graphs
                               whose visited sets fit in shared memory, whose nodes have at most 8 out-roads
                               and that have no road from a node to itself: a walk still going after this
                               many moves is suspended and finished by a pipelined kernel with one ant per
                               warp (the same walks, sooner); 0 = off; ignored where it does not apply */
} gmp_params;

/* Pheromone layouts. Dense: every road's pheromone is evaporated every iteration. Sparse: roads that never
 * received a deposit all hold one value per colony (the baseline, evaporated once per iteration) and only
 * roads with deposits are evaporated one by one; iterative mode with the constant initial pheromone only.
 * AUTO takes sparse for graphs of at least 65536 roads when it applies, dense otherwise. */
#define GMP_TAU_AUTO 0u
#define GMP_TAU_DENSE 1u
#define GMP_TAU_SPARSE 2u

/* One origin-destination colony. alpha, beta in [0, 8]: integers score f^alpha * (1/c)^beta by repeated
 * binary32 multiplication; other values score 2^(alpha log2 f - beta log2 c) with the library's own
 * binary32 log2 and exp2 (within 2^-21 (alpha |log2 f| + beta log2 c + 1) relative of the exact power).
 * rho in [0, 1). */
typedef struct {
    uint32_t src, dst, n_ants, n_iter;
    float alpha, beta, rho;
    uint32_t reserved;
    uint64_t seed;
} gmp_query;

/* Result of one colony. `route` is a caller-owned buffer of `route_cap` node ids. */
typedef struct {
    uint32_t *route;    /* best route as node ids, src first, dst last */
    uint32_t route_cap; /* capacity of `route` in entries */
    uint32_t route_len; /* nodes in the best route (required size if status == GMP_ERR_BUFFER) */
    uint64_t travel_ms; /* T of the best route: min T over all ants, ties to lowest (iteration, ant) */
    uint64_t wait_ms;   /* signal waits + queue delays along that route */
    uint64_t ant_steps; /* moves of all ants of all iterations (forward and back), failed ants included */
    uint64_t n_success; /* ant walks that reached the destination */
    uint32_t best_iter, best_ant;
    int32_t status;     /* GMP_OK, GMP_ERR_NO_ROUTE or GMP_ERR_BUFFER */
    uint32_t reserved;
} gmp_result;

/* Create a context on CUDA device `device`. mem_budget_bytes bounds the device memory the context may
 * hold (0 = no bound). cuda_stream is a cudaStream_t to issue work on (NULL = a stream the context owns).
 * Errors: INVALID_ARG (bad device), CUDA. */
int gmp_create(gmp_ctx **out, int device, uint64_t mem_budget_bytes, void *cuda_stream);

/* Release every device allocation of the context. NULL is ignored. */
void gmp_destroy(gmp_ctx *ctx);

/* Human-readable name of a return code. Static storage. */
const char *gmp_strerror(int code);

/* Last detailed error message of the context (static storage inside the context). */
const char *gmp_last_error(const gmp_ctx *ctx);

/* Issue subsequent work on cuda_stream (NULL = the context's own stream). */
int gmp_set_stream(gmp_ctx *ctx, void *cuda_stream);

/* Optional: place every device allocation of the context (graph, traffic state, batch workspace) inside
 * caller-owned device memory [dev_ptr, dev_ptr + bytes), for example a tensor from the caller's allocator,
 * instead of cudaMalloc. Call it before gmp_load_graph. The memory must be 256-byte aligned device memory
 * of the context's GPU and stay valid, and untouched by the caller, until gmp_destroy; the library never
 * frees it. Allocations are first fit in 256-byte multiples with free runs merged. A request that does
 * not fit fails with GMP_ERR_OOM, and the memory budget of gmp_create still applies. dev_ptr == NULL
 * unbinds (also only before gmp_load_graph). Errors: INVALID_ARG (alignment, size, not device memory of
 * this GPU), STATE (the context already holds device memory). */
int gmp_bind_workspace(gmp_ctx *ctx, void *dev_ptr, uint64_t bytes);

/* Make ctx a view of owner's road graph: ctx reads owner's static arrays (topology, road attributes,
 * coordinates, signal programmes) in place, without a copy, and with own_state = 0 also owner's traffic
 * state (vehicles, red times, phase order, road records); with own_state = 1 it gets a copy of that
 * state which it may change (gmp_set_densities, gmp_set_red_times, gmp_tick) without touching owner's.
 * ctx keeps its own parameters, stream and batch workspace, and drops whatever graph it held before. A
 * view cannot change the signal programmes, nor (with own_state = 0) the traffic state, its threshold or
 * headway (GMP_ERR_STATE). owner must outlive its views; while it has views it cannot load another graph
 * or change its signals (GMP_ERR_STATE), and changes to its traffic state reach views that share it.
 * Synchronous. The paper has no counterpart (a server's slots share one graph this way).
 * Errors: INVALID_ARG (same context, other device), STATE (owner holds no graph, ctx has views), OOM,
 * CUDA. */
int gmp_share_graph(gmp_ctx *ctx, gmp_ctx *owner, int own_state);

/* Road graph G(N, E) (the graph of Fig. 3; Sec. 5: roads with lanes) in CSR form: the roads leaving
 * node u are row_ptr[u] .. row_ptr[u+1]-1, in the order that breaks ties between equal choices.
 * col[e]: head node; length_dm[e] >= 1; speed_kmh[e] >= 1; lanes[e] >= 1; x_dm, y_dm: node coordinates,
 * |x|, |y| <= 2^27. Derives free-flow times and jam capacities on the device. Replaces any previous graph
 * and resets signals (none) and densities (zero). Errors: INVALID_ARG, OOM, CUDA. */
int gmp_load_graph(gmp_ctx *ctx, uint32_t n_nodes, uint32_t n_edges, const uint32_t *row_ptr, const uint32_t *col,
                   const uint32_t *length_dm, const uint16_t *speed_kmh, const uint8_t *lanes, const int32_t *x_dm,
                   const int32_t *y_dm);

/* Fixed-time signal programmes (the lights and phases of Fig. 3; Algorithm 1 arguments traffic_light, phases).
 * Per node v: n_phases[v] in 0..8 (0 = unsignalised), cycle_ms[v] in 1..2^24-1, offset_ms[v] < cycle,
 * green_ms[v*8 + p] >= 1 for p < n_phases with sum == cycle. edge_phase[e]: approach phase of road e at
 * its head (< n_phases of the head when signalised). Resets the red-time accumulators to 0 and recomputes
 * the phase order. Errors: INVALID_ARG, UNSUPPORTED (> 8 phases), STATE (no graph), CUDA. */
int gmp_set_signals(gmp_ctx *ctx, const uint8_t *n_phases, const uint32_t *cycle_ms, const uint32_t *offset_ms,
                    const uint32_t *green_ms, const uint8_t *edge_phase);

/* Red-time accumulators t_p of Fig. 3 (how long each phase's vehicles have waited), host array of N*8
 * entries in ms (node*8 + phase; entries at or above a node's phase count do not enter the order), copied by the
 * call. Recomputes the phase order on the device. Synchronous. Errors: INVALID_ARG, STATE (no graph),
 * CUDA. */
int gmp_set_red_times(gmp_ctx *ctx, const uint32_t *red_ms);

/* Vehicles currently on each road (Sec. 4.2: densities from road sensors; Calc_Dens). Recomputes edge
 * travel times, queue delays and the phase order on the device. Host array of E entries.
 * Errors: STATE, CUDA. */
int gmp_set_densities(gmp_ctx *ctx, const uint32_t *vehicles);

/* Same from device memory (E entries of the context's GPU), asynchronous on the context's stream: the
 * caller keeps d_vehicles unchanged until that stream has passed the call. Errors: INVALID_ARG, STATE,
 * CUDA. */
int gmp_set_densities_async(gmp_ctx *ctx, const uint32_t *d_vehicles);

/* Read back the vehicles on each road (host array of E entries) and the red-time accumulators (host
 * array of N*8 entries, ms), as the last density update or tick left them. Synchronous.
 * Errors: INVALID_ARG, STATE, CUDA. */
int gmp_get_densities(gmp_ctx *ctx, uint32_t *vehicles);
int gmp_get_red_times(gmp_ctx *ctx, uint32_t *red_ms);

/* Serving tick: advances the traffic state held by the context by dt_ms at clock t_now_ms (the queue and
 * preemption update of the Fig. 3 signal block, Calc_Dens / Comp_Thres of Sec. 4.2, with vehicles
 * that move). In order:
 *   - the phase green at t_now_ms under each node's current phase order (windows laid out from the
 *     node's offset); every approach of an unsignalised node is served;
 *   - each served road discharges min(n, c) vehicles, c = lanes*(t_now+dt)/h_sat - lanes*t_now/h_sat
 *     in integer division (the saturation flow counted on the whole clock);
 *   - a node's discharge K goes to its d out-roads, K/d each and one more to each of the first K mod d
 *     in CSR order; vehicles reaching a node without out-roads leave the network; counts are 32-bit
 *     and wrap as unsigned arithmetic;
 *   - red-time accumulators: 0 for the green phase and for phases whose approaches are empty before the
 *     discharge, + dt_ms (saturating at 2^32-1) for the others;
 *   - road travel times, queue delays and the phase order are recomputed from the new state.
 * Asynchronous on the context's stream: it is ordered after any job already launched there and before
 * any launched later. Requires t_now_ms <= 2^48 and dt_ms <= 2^30. Its scratch (E*4 + N*8 bytes) is
 * allocated with the graph. Errors: INVALID_ARG, STATE, CUDA. */
int gmp_tick(gmp_ctx *ctx, uint64_t t_now_ms, uint32_t dt_ms);

/* Schedule chosen by gmp_autotune. */
typedef struct {
    uint32_t lanes_per_ant; /* lanes of a warp per ant (ants per warp = 32 / lanes; 1 = one thread per ant) */
    uint32_t mode;          /* GMP_MODE_ITERATIVE or GMP_MODE_PERSISTENT */
    uint32_t queue_chunk;   /* persistent mode: intersections per queue-update work item; 0 otherwise */
    uint32_t lockstep;      /* 1 when the ants of a warp step together (iterative mode) */
    uint32_t branches;      /* iterative mode: concurrent colony chains (0 = the default) */
    uint32_t from_cache;    /* 1 when this size bucket was tuned earlier in the process: nothing was timed */
    uint32_t n_tried;       /* schedules timed */
    float best_ms;          /* probe job time of the chosen schedule (0 from the cache) */
    float default_ms;       /* probe job time of the untuned schedule (0 from the cache) */
    uint32_t bucket[4];     /* size bucket: SM count, ceil(log2 N), max out-degree, ceil(log2 probe ants) */
    uint32_t handoff_moves; /* iterative mode: moves after which a walk is handed to the tail kernel (0 = off) */
} gmp_tune_result;

/* Autotuner for the batched job (no counterpart in the paper, whose kernels have one fixed shape). All
 * schedules give the same results bit for bit, so only speed differs. The first call for a size bucket
 * times a probe job (the n probe queries with n_iter clamped to probe_iter, 0 = 8) under every schedule
 * the graph admits: lanes per ant 1/4/8/16/32, warp lockstep or free-running groups, the iterative or
 * the persistent job with queue chunks 8/16/32/64, free-running groups that hand walks longer than 512
 * moves to the tail kernel (where gmp_params.handoff_moves applies), and then, for the best iterative
 * schedule, 1, 4, 32 or 64 concurrent colony chains instead of the default and, if it hands walks off,
 * 256 or 2048 moves instead of 512. Each is run once to warm up, then twice timed on
 * the context's stream (best of two); the untuned schedule is timed first and a schedule replaces the
 * best so far only when it is at least 3% faster. The choice is cached for the process by bucket and written
 * into the context's parameters (lanes_per_ant, mode, queue_chunk, branches, handoff_moves, the lockstep
 * flag); later calls in
 * the same bucket apply the cached choice without timing. Replaces any staged batch. Synchronous.
 * Errors: INVALID_ARG, STATE, UNSUPPORTED (no schedule ran), and those of gmp_batch_stage. */
int gmp_autotune(gmp_ctx *ctx, uint32_t n, const gmp_query *probe, uint32_t probe_iter, gmp_tune_result *out);

/* Forget every cached autotuner choice of the process. */
void gmp_autotune_reset(void);

/* ---------------------------------------------------------------------------------------------- */
/* Many road graphs in one launch (the ragged multi-graph batch; the paper solves one graph).         */
/* ---------------------------------------------------------------------------------------------- */
typedef struct gmp_multi gmp_multi;

/* A handle that launches the staged jobs of several contexts (each holding its own road graph, on the
 * handle's device) as one captured CUDA graph on a stream of its own. Errors: INVALID_ARG, CUDA. */
int gmp_multi_create(gmp_multi **out, int device);
void gmp_multi_destroy(gmp_multi *multi);
const char *gmp_multi_last_error(const gmp_multi *multi);

/* Launch the batches staged on ctxs[0..n) (gmp_batch_stage on each first; iterative mode) together: one
 * fork per context into its own concurrent colony chains, one join, one graph launch. The capture is kept
 * and replayed while the same contexts keep batches of the same shape. The launch is ordered after work
 * already queued on every context's stream, and every context's stream is ordered after the launch, so
 * gmp_batch_ready and gmp_batch_collect are then used per context as after gmp_batch_launch. Each result
 * equals that of its batch launched alone. Asynchronous. A context may appear once.
 * Errors: INVALID_ARG, STATE (a context without a staged batch), UNSUPPORTED (persistent mode), CUDA. */
int gmp_multi_launch(gmp_multi *multi, gmp_ctx *const *ctxs, uint32_t n);

/* ---------------------------------------------------------------------------------------------- */
/* Route server: continuous batching over several contexts (no counterpart in the paper, which routes */
/* one vehicle at a time in Fig. 3).                                                                  */
/* ---------------------------------------------------------------------------------------------- */
typedef struct gmp_server gmp_server;

typedef struct {
    uint32_t max_batch;      /* requests per job at most (memory may admit fewer) */
    uint32_t max_ants;       /* largest n_ants a request may ask for */
    uint32_t max_iter;       /* largest n_iter a request may ask for */
    uint32_t mem_budget_mib; /* device memory all slots' batch workspaces may hold together, in MiB; 0 = no
                                bound beyond the memory the GPU has free */
} gmp_server_config;

/* One finished request. Times are host steady-clock nanoseconds. */
typedef struct {
    uint64_t tag;         /* the caller's id from gmp_server_submit */
    uint64_t t_submit_ns; /* submitted */
    uint64_t t_launch_ns; /* its job was launched */
    uint64_t t_done_ns;   /* the server saw its job finished (at a gmp_server_pump) */
    uint64_t clock_ms;    /* traffic clock of the state it was solved on: t_now + dt of the last tick
                             issued before its job (0 before any tick) */
    uint32_t slot;        /* the slot that ran it */
    uint32_t batch_size;  /* requests in that job */
    gmp_result result;    /* route points into the buffer given to gmp_server_take; status as for
                             gmp_batch_collect, or the error that failed the whole job */
} gmp_served;

typedef struct {
    uint32_t queued;       /* waiting for a slot */
    uint32_t in_flight;    /* in jobs on the GPU */
    uint32_t busy_slots;   /* slots with a job on the GPU */
    uint32_t done_waiting; /* finished, not yet taken */
    uint64_t jobs;         /* jobs launched so far */
    uint64_t completed;    /* requests finished so far */
    uint64_t rejected;     /* requests refused at submission */
} gmp_server_stats;

/* Create a server with n_slots slots over the road graph of `graph` (a context holding the loaded graph,
 * signals, densities, red times and parameters, with a traffic state of its own). The slots are views of
 * that graph (gmp_share_graph): its static arrays exist once on the GPU. The server keeps two versions of
 * the traffic state, graph's own and a copy of its own, so that a tick never stops running jobs (see
 * gmp_server_tick). Each slot has a batch workspace and a CUDA stream of its own; workspaces grow through
 * the stream-ordered allocator. graph must outlive the server and must not be changed while it exists
 * (the server changes its traffic state at ticks). Admission is per job: an idle slot takes up to
 * max_batch requests from the head of the queue, fewer when their workspace would not fit the server's
 * memory budget together with the other slots' workspaces, or the memory the GPU has free; requests that
 * do not fit wait. Errors: INVALID_ARG, STATE (no graph, or graph reads another context's state), OOM,
 * CUDA. */
int gmp_server_create(gmp_server **out, gmp_ctx *graph, uint32_t n_slots, const gmp_server_config *cfg);
void gmp_server_destroy(gmp_server *srv);
const char *gmp_server_last_error(const gmp_server *srv);

/* Device memory the slots' batch workspaces hold together, and the server's budget (0 = none). */
int gmp_server_memory(const gmp_server *srv, uint64_t *slots_bytes, uint64_t *budget_bytes);

/* Queue one request (FIFO). Checked at once: a request that a job would refuse, or one above max_ants
 * or max_iter, is refused here with that error and counted as rejected. */
int gmp_server_submit(gmp_server *srv, const gmp_query *query, uint64_t tag);

/* Advance the traffic state by one tick gmp_tick(t_now_ms, dt_ms): the server copies the current version
 * of the state into the other one and ticks that copy, on its own stream, after the jobs still reading
 * the version it overwrites (those launched before the previous tick); running jobs on the current
 * version are not waited for. Jobs launched afterwards run on the new version, after the tick, and depart
 * at the new serving clock t_now_ms + dt_ms (the server sets the slot's t_dep_ms), so the clock must stay
 * below 2^30 ms. Asynchronous. Errors: INVALID_ARG, CUDA, and those of gmp_tick. */
int gmp_server_tick(gmp_server *srv, uint64_t t_now_ms, uint32_t dt_ms);

/* One non-blocking round of the loop: collect every job that has finished, then give every idle slot
 * the requests waiting at the head of the queue (up to its admission limit) as one job and launch it.
 * Fills *stats when non-NULL. */
int gmp_server_pump(gmp_server *srv, gmp_server_stats *stats);

/* Move up to max_n finished requests, oldest first, into out[]; their routes are copied back to back into
 * route_buf (route_entries entries). Stops early when the next route does not fit.
 * Errors: INVALID_ARG, BUFFER (not even the first route fits). */
int gmp_server_take(gmp_server *srv, uint32_t max_n, gmp_served *out, uint32_t *route_buf, uint64_t route_entries,
                    uint32_t *n_out);

/* Colony tunables; recomputes threshold flags. Errors: INVALID_ARG. */
int gmp_set_params(gmp_ctx *ctx, const gmp_params *params);
int gmp_get_params(const gmp_ctx *ctx, gmp_params *params);

/* One colony (Algorithm 2 for one origin-destination pair): n_iter iterations of n_ants ants each,
 * then the best route. Each ant (Fig. 3's body for one vehicle) starts at src with a visited set; at each
 * node it draws the next road among those leading to unvisited nodes by a roulette over tau^alpha *
 * (1/c)^beta, c = the time the road adds over the remaining lower bound (travel time + signal wait and
 * queue delay at its head + h(head) - h(here), at least 1 ms). At a node with no such road it steps
 * back to the previous node of its route (whose clock and wait come back; the node it left stays
 * visited). It ends at dst, back at src with nothing left, after max_steps moves, or past 2^30 ms.
 * Synchronous; equivalent to gmp_solve_batch with one query.
 * Errors: INVALID_ARG, UNSUPPORTED, STATE, OOM, CUDA, TIMEOUT; NO_ROUTE / BUFFER via out->status too. */
int gmp_solve(gmp_ctx *ctx, uint32_t src, uint32_t dst, uint32_t n_ants, uint32_t n_iter, float alpha, float beta,
              float rho, uint64_t seed, gmp_result *out);

/* n independent colonies on the context's graph in one device job (queries may differ in ants and
 * iterations). Each result equals that of the query solved alone. Synchronous; host queries and results.
 * Returns GMP_OK when the job ran (per-query outcomes in results[i].status), else an error code. */
int gmp_solve_batch(gmp_ctx *ctx, uint32_t n, const gmp_query *queries, gmp_result *results);

/* The three phases of gmp_solve_batch, for callers that keep inputs and outputs on the device:
 *   gmp_batch_stage   validates and uploads n queries (host array, copied), reserves the device
 *                     workspace (synchronous). Errors: INVALID_ARG, UNSUPPORTED, STATE, OOM, CUDA;
 *   gmp_batch_launch  issues the whole job on the stream and returns (no host synchronisation, no copies).
 *                     Errors: INVALID_ARG, STATE (nothing staged), CUDA;
 *   gmp_batch_collect waits for the job and copies results[0..n) back (host array of n; routes into the
 *                     buffers each result names). Errors: INVALID_ARG, STATE (nothing launched), TIMEOUT
 *                     (a bounded device wait expired), CUDA.
 * gmp_batch_launch may be called repeatedly on a staged batch; every launch starts from fresh pheromone. */
int gmp_batch_stage(gmp_ctx *ctx, uint32_t n, const gmp_query *queries);
int gmp_batch_launch(gmp_ctx *ctx);
int gmp_batch_collect(gmp_ctx *ctx, gmp_result *results);

/* Reserve the device workspace of the largest job the caller will stage: n colonies, total_ants ants
 * per iteration (summed over the colonies), up to max_iter iterations, under the current parameters
 * (lanes, mode, ant log). Buffers only grow, so staging any job within these bounds afterwards allocates
 * nothing (and so never waits on the allocator while jobs of other contexts run). Drops any staged
 * batch; on OOM the whole workspace is released. Synchronous.
 * Errors: INVALID_ARG, STATE, UNSUPPORTED, OOM (the memory budget or the device cannot hold it), CUDA. */
int gmp_batch_reserve(gmp_ctx *ctx, uint32_t n, uint64_t total_ants, uint32_t max_iter);

/* Non-blocking: *ready = 1 when the last launched job has finished on the device, else 0.
 * Errors: INVALID_ARG, STATE (nothing launched), CUDA (the job failed). */
int gmp_batch_ready(gmp_ctx *ctx, int *ready);

/* Pheromone of query `slot` of the last batch after its final iteration: host array of E entries, Q32.32
 * (rebuilt from the baseline and the registered roads in the sparse layout). Synchronous.
 * Errors: INVALID_ARG (slot out of range), STATE (no batch ran), OOM, CUDA. */
int gmp_get_pheromone(gmp_ctx *ctx, uint32_t slot, uint64_t *out_tau);

/* Per-(iteration, ant) log of query `slot` (needs GMP_FLAG_ANT_LOG when the batch ran):
 * n_iter*n_ants*4 entries {status | roads in the route << 8, moves, T, W}; status 0 success, 1 dead end
 * (back at src with no road left), 2 step cap, 3 time cap.
 * Host array of capacity_entries. Errors: INVALID_ARG, STATE (no log), BUFFER (capacity too small), CUDA. */
int gmp_get_ant_log(gmp_ctx *ctx, uint32_t slot, uint32_t *out, uint64_t capacity_entries);

/* Current per-node phase order (host array of N*8 entries; positions >= n_phases hold p) -- the
 * preemptive plan. Synchronous. Errors: INVALID_ARG, STATE (no graph), CUDA. */
int gmp_get_phase_order(gmp_ctx *ctx, uint8_t *out);

/* Current congested travel time and queue delay per road (host arrays of E entries each; either may be
 * NULL). Synchronous. Errors: INVALID_ARG, STATE (no graph), CUDA. */
int gmp_get_edge_times(gmp_ctx *ctx, uint32_t *tt_ms, uint32_t *qd_ms);

/* Device time of the last launched job (staged with the per-kernel timing flag), in ms: out[0] construction,
 * out[1] iteration end (evaporation + deposit, best-route tracking and queue/preemption in one kernel),
 * both summed over the concurrent colony chains (which overlap in time), out[2] initialisation + result
 * rows, out[3] 0, out[4] whole job. In the persistent job everything but initialisation and the result
 * rows is one kernel, reported as out[0]. Waits for the stream. Errors: INVALID_ARG, STATE (no job staged with
 * the timing flag has run), CUDA. */
int gmp_get_kernel_times(gmp_ctx *ctx, float *out_ms5);

/* Count of kernel launches issued by the last gmp_batch_launch. */
int gmp_get_launch_count(const gmp_ctx *ctx, uint64_t *out);

/* Result row written to device memory by gmp_solve_static (the same fields as gmp_result, without the
 * route buffer; status GMP_OK or GMP_ERR_NO_ROUTE; route_len counts nodes). */
typedef struct {
    uint64_t travel_ms, wait_ms, ant_steps, n_success;
    uint32_t route_len, best_iter, best_ant;
    int32_t status;
} gmp_device_result;

/* Size of the library's static scratch array used by gmp_solve_static. */
#define GMP_STATIC_SCRATCH_BYTES ((uint64_t)32 << 20)

/* One colony on the context's graph that allocates no device memory during the call. The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc while they solve (a loop that must never
 * wait on the allocator, an exhausted memory pool or quota, a framework that owns every allocation).
 * Every temporary lives in a device array of GMP_STATIC_SCRATCH_BYTES that the library defines at file
 * scope; the caller passes the outputs: d_result (one row) and d_route (route_cap >= min(N, max_steps + 1)
 * entries, the nodes of the longest possible route), both device memory of the context's GPU. The work is issued on the context's stream and
 * the call returns without waiting; synchronise that stream before reading the outputs. The first call
 * on a device looks the array's address up, so make it before any stream capture. Every call reuses the
 * same array (which keeps the previous call's data; each call re-initialises what it needs), so calls
 * that overlap on the GPU race. The colony runs like gmp_solve (same results, the ant log excepted),
 * always in the dense pheromone layout (both layouts give the same results, so tau_layout is not read),
 * in warp lockstep unless the context's parameters turn lockstep off.
 * Errors: INVALID_ARG, UNSUPPORTED, STATE, CUDA; BUFFER when route_cap is short or when the colony's
 * temporaries (about 24 bytes per road plus 8 * n_ants * max_steps bytes) exceed the array. */
int gmp_solve_static(gmp_ctx *ctx, uint32_t src, uint32_t dst, uint32_t n_ants, uint32_t n_iter, float alpha,
                     float beta, float rho, uint64_t seed, gmp_device_result *d_result, uint32_t *d_route,
                     uint32_t route_cap);

#ifdef __cplusplus
}
#endif

#endif /* GMACOP_H */

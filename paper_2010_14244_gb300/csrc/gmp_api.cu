// C ABI of libgmacop.so (declared and documented in include/gmacop.h).
//
// Replaces the paper's Algorithm 1 (allocate, copy in, one launch, copy out, free per call) with a
// context that keeps the graph, signals, densities and batch workspace resident on the GPU, and a
// whole colony job (init, then per iteration: construction, evaporation+deposit, best tracking,
// queue/preemption update; then the result rows) captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "gmacop.h"
#include "gmp_internal.h"

using namespace gmp;

namespace {

constexpr uint32_t kFlagKernelTiming = 4u;  // event records around every kernel of the job
constexpr uint32_t kFlagNoGraph = kFlagNoGraphBit;  // issue the job kernel by kernel instead of replaying a graph
constexpr uint32_t kFlagNoLockstep = kFlagNoLockstepBit;  // sub-warp ants without warp lockstep
constexpr uint32_t kKnownFlags =
    GMP_FLAG_RANDOM_TAU | GMP_FLAG_ANT_LOG | GMP_FLAG_PAPER_LITERAL | GMP_FLAG_EXACT_H | kFlagKernelTiming | kFlagNoGraph |
    kFlagNoLockstep;
constexpr int32_t kCoordLimit = 1 << 27;
constexpr uint64_t kTickClockMax = 1ull << 48;  // lanes * (t + dt) stays below 2^64
constexpr uint32_t kDefaultBranches = 16;        // concurrent colony chains of an iterative job
constexpr size_t kMaxCachedGraphs = 32;          // executable graphs kept per context, by topology
constexpr uint32_t kSparseMinEdges = 1u << 16;   // GMP_TAU_AUTO: sparse pheromone from this many roads
constexpr uint32_t kMaxBranches = 64;
constexpr uint32_t kTickDtMax = 1u << 30;

struct BatchKey {
    uint32_t Q = 0, maxI = 0, total_ants = 0, max_steps = 0, flags = 0, lanes = 0, grid = 0, thr_on = 0, t_dep = 0,
             chunk = 0, branches = 0, sparse = 0, poll_limit = 0, level_limit = 0, handoff = 0;
    uint64_t log_entries = 0;
    const void* ptrs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool operator==(const BatchKey& o) const { return memcmp(this, &o, sizeof(BatchKey)) == 0; }
};

struct Batch {
    uint32_t Q = 0, maxI = 0, total_ants = 0, max_steps = 0;
    uint64_t log_entries = 0;
    std::vector<gmp_query> hq;
    bool staged = false, ran = false;
    bool dep_dirty = false;  // the deposit accumulators may hold a stopped job's deposits
    KernelConfig kc{};
    // device workspace
    DevQuery* dq = nullptr;
    uint32_t* prefix = nullptr;
    uint64_t* tau = nullptr;      // dense layout: Q * E
    bool sparse = false;          // sparse layout: baseline + registered roads (see EdgeRec notes)
    uint32_t* tflag = nullptr;    // sparse: Q * tflag_words registered-road bitmap
    uint32_t* list_e = nullptr;   // sparse: Q * E registered roads
    uint64_t* list_tau = nullptr; // sparse: Q * E their pheromone
    uint2* th = nullptr;  // per (colony, road): pheromone as binary32 bits, heuristic (ms)
    unsigned long long* dep = nullptr;
    QueryState* qs = nullptr;
    uint32_t* routes = nullptr;
    uint32_t* ant_steps = nullptr;
    uint32_t* ant_wait = nullptr;
    uint32_t* best_route = nullptr;
    uint32_t* route_out = nullptr;
    uint32_t* tickets = nullptr;
    uint32_t* ant_log = nullptr;
    uint32_t* tabu = nullptr;
    DevResult* res = nullptr;
    // hand-off of long walks to the tail kernel (handoff: the move count, 0 = off for this job)
    uint32_t handoff = 0;
    uint32_t* tail_list = nullptr;    // total_ants: suspended walks, per chain from its first ant on
    WalkState* tail_state = nullptr;  // total_ants
    uint32_t* tail_tabu = nullptr;    // total_ants * visited-bitmap words
    // persistent job
    bool persistent = false;
    IterCounters* ctr = nullptr;
    uint32_t* qstate = nullptr;
    uint32_t* qflag = nullptr;
    uint32_t* misc = nullptr;  // [0] finished colonies, [1] persistent wait expired, [2] exact-h level bound
    bool queue_general = false;  // intersections with more than two phases: a queue pass of their own
    // exact Calc_Dist (GMP_FLAG_EXACT_H)
    bool exact_h = false;
    uint32_t* hdist = nullptr;   // Q * N bounds
    uint32_t* hqueue = nullptr;  // Q * 4N: near frontiers (2N) and far piles (2N)
    uint32_t* hstamp = nullptr;  // Q * 2N: near (per level) and far (per epoch) stamps
    // captured job
    cudaGraphExec_t exec = nullptr;  // the executable graph of the staged job (one of `execs`)
    std::map<std::vector<uint32_t>, cudaGraphExec_t> execs;  // by topology, refreshed by graph update
    BatchKey key{};
    uint64_t launches = 0;
    std::vector<cudaEvent_t> ev;
    bool timed = false;
    cudaEvent_t done = nullptr;  // recorded after every launch (gmp_batch_ready)
    // iterative job: contiguous colony ranges run as concurrent chains of launches
    struct Branch {
        uint32_t q0, q1, ants, ticket_base, maxI;
        KernelConfig kc;
        KernelConfig kc_tail;  // the tail kernel of this chain (hand-off)
        size_t tabu_off;  // words into the global visited-bitmap pool
    };
    std::vector<Branch> br;
    std::vector<Branch> exec_br;  // the chain plan baked into `exec`
    size_t tabu_used = 0;         // words of the global visited-bitmap pool this job uses
};

// What fixes the node structure of a captured job: the job form, timing events, the chains with their
// iteration counts and kernel shapes. Jobs with equal topology differ only in kernel parameters.
std::vector<uint32_t> topology_of(const Batch& b) {
    std::vector<uint32_t> t{b.persistent ? 1u : 0u, b.timed ? 1u : 0u, b.exact_h ? 1u : 0u, b.queue_general ? 1u : 0u,
                            b.handoff ? 1u : 0u,
                            (uint32_t)b.br.size(), b.maxI,
                            (uint32_t)b.kc.lanes, (uint32_t)b.kc.slots, b.kc.lockstep ? 1u : 0u,
                            b.kc.tabu_in_smem ? 1u : 0u, (uint32_t)b.kc.block, b.kc.frac ? 1u : 0u};
    for (const Batch::Branch& r : b.br) {
        t.push_back(r.maxI);
        t.push_back((uint32_t)r.kc.lanes | (uint32_t)r.kc.slots << 8 | (r.kc.lockstep ? 1u << 16 : 0u) |
                    (r.kc.tabu_in_smem ? 1u << 17 : 0u) | (r.kc.frac ? 1u << 18 : 0u));
        t.push_back((uint32_t)r.kc.block);
    }
    return t;
}

bool same_plan(const std::vector<Batch::Branch>& x, const std::vector<Batch::Branch>& y) {
    if (x.size() != y.size()) return false;
    for (size_t i = 0; i < x.size(); ++i) {
        const Batch::Branch &a = x[i], &b = y[i];
        if (a.q0 != b.q0 || a.q1 != b.q1 || a.ants != b.ants || a.ticket_base != b.ticket_base || a.maxI != b.maxI ||
            a.tabu_off != b.tabu_off || a.kc.grid != b.kc.grid || a.kc.block != b.kc.block ||
            a.kc.lanes != b.kc.lanes || a.kc.slots != b.kc.slots || a.kc.smem != b.kc.smem ||
            a.kc.tabu_in_smem != b.kc.tabu_in_smem || a.kc.lockstep != b.kc.lockstep || a.kc.frac != b.kc.frac ||
            a.kc_tail.grid != b.kc_tail.grid || a.kc_tail.smem != b.kc_tail.smem)
            return false;
    }
    return true;
}

}  // namespace

struct gmp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    uint64_t budget = 0, used = 0;
    std::unordered_map<void*, size_t> sizes;
    // caller-owned device memory (gmp_bind_workspace): allocations are carved from it instead of cudaMalloc
    char* arena = nullptr;
    uint64_t arena_bytes = 0;
    std::map<uint64_t, uint64_t> arena_free;           // offset -> length of each free run
    std::unordered_map<void*, uint64_t> arena_blocks;  // allocation -> length carved for it
    std::string err;
    gmp_params prm{};
    bool has_graph = false;
    uint32_t N = 0, E = 0, maxdeg = 0, kappa = 0;
    uint32_t h_delta = 1;  // exact heuristic: near-far threshold step, 16 x the mean free-flow road time (ms)
    uint32_t max_phases = 0;  // most phases at any intersection (above 2: the iteration end's general pass)
    bool self_loops = false;  // some road leads from a node back to itself
    uint32_t *row_ptr = nullptr, *col = nullptr, *len = nullptr, *in_ptr = nullptr, *in_edge = nullptr;
    uint32_t* in_tail = nullptr;  // tail of each in_edge entry (exact Calc_Dist relaxes towards tails)
    // Per-approach tables are in slot order (slot i = road in_edge[i], so an intersection's approaches
    // are contiguous); phase tables are phase-major (entry p * N + v). The C ABI speaks road order and
    // node-major phase rows; the calls that take or return those tables convert.
    uint32_t *ff = nullptr, *cap = nullptr;  // per slot: free-flow time, jam capacity
    uint16_t* speed = nullptr;
    uint8_t* lanes = nullptr;     // per road
    uint8_t* lanes_in = nullptr;  // per slot
    int32_t *x = nullptr, *y = nullptr;
    uint8_t *nph = nullptr, *ephase = nullptr, *order = nullptr;  // ephase per slot, order node-major
    uint32_t *cycle = nullptr, *offset = nullptr, *green = nullptr, *red = nullptr;  // green, red phase-major
    uint32_t* veh = nullptr;      // per slot
    bool red_high = false;        // red planes at or above max_phases may hold non-zero values
    EdgeRec* rec = nullptr;
    uint32_t* tick_leave = nullptr;        // serving tick: discharge of each slot (E); density upload scratch
    unsigned long long* tick_K = nullptr;  // serving tick: discharge of each node (N)
    std::vector<int32_t> hx, hy;  // host copy of node coordinates (destination lookups at staging)
    std::shared_ptr<const std::vector<uint32_t>> hin_edge;  // host copy of in_edge (road-order conversions)
    // A context may view another context's road graph (gmp_share_graph): the static arrays always, the
    // traffic state (vehicles, red times, phase order, road records, tick scratch) too unless it keeps a
    // state of its own. What a view borrowed is never freed by it.
    gmp_ctx* lender = nullptr;        // owner of the static arrays, or nullptr
    gmp_ctx* state_lender = nullptr;  // holder of the traffic state this context reads, or nullptr (own)
    bool own_state = true;            // the traffic-state arrays are this context's allocations
    int views = 0;                    // contexts that borrow this context's static arrays or state
    bool stream_alloc = false;        // device memory from the stream-ordered allocator on `stream` (no
                                      // device-wide synchronisation when a workspace grows)
    Batch b;
    std::vector<cudaStream_t> bstreams;  // streams of the concurrent colony chains
    std::vector<cudaEvent_t> bjoin;      // one join event per chain
    cudaEvent_t bfork = nullptr;
};

namespace gmp {

uint32_t default_lanes(uint32_t maxdeg) {
    for (uint32_t g : {8u, 16u, 32u})  // one candidate slot per lane when the degree allows
        if (g >= maxdeg) return g;
    return 32u;
}

bool lockstep_fits(int lanes, uint32_t maxdeg) {
    if (lanes == 1) return true;  // one thread per ant always steps in lockstep
    return lanes <= 16 && maxdeg <= (uint32_t)(2 * lanes) && lanes * (maxdeg <= (uint32_t)lanes ? 1 : 2) <= 16;
}

CtxInfo ctx_info(const gmp_ctx* c) {
    return CtxInfo{c->device, c->stream, c->N, c->E, c->maxdeg, c->has_graph, c->budget, c->used};
}

int ctx_fail(gmp_ctx* c, int code, const char* msg) {
    if (c) c->err = msg;
    return code;
}

}  // namespace gmp

namespace {

int fail(gmp_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define GMP_CUDA(c, call)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((c), GMP_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define GMP_TRY(x)             \
    do {                       \
        int r_ = (x);          \
        if (r_ != GMP_OK) return r_; \
    } while (0)

// First fit in the bound workspace: runs of 256-byte multiples, split on allocation.
void* arena_take(gmp_ctx* c, size_t bytes) {
    const uint64_t need = ((uint64_t)bytes + 255u) & ~(uint64_t)255u;
    for (auto it = c->arena_free.begin(); it != c->arena_free.end(); ++it) {
        if (it->second < need) continue;
        const uint64_t off = it->first, len = it->second;
        c->arena_free.erase(it);
        if (len > need) c->arena_free[off + need] = len - need;
        void* q = c->arena + off;
        c->arena_blocks[q] = need;
        return q;
    }
    return nullptr;
}

// Return a block to the bound workspace, merging it with free neighbours. Like cudaFree, it first waits
// for the context's work (every job joins its chains back into the context's stream).
void arena_give(gmp_ctx* c, void* q) {
    cudaStreamSynchronize(c->stream);
    auto b = c->arena_blocks.find(q);
    if (b == c->arena_blocks.end()) return;
    uint64_t off = (uint64_t)((char*)q - c->arena), len = b->second;
    c->arena_blocks.erase(b);
    auto next = c->arena_free.lower_bound(off);
    if (next != c->arena_free.end() && next->first == off + len) {
        len += next->second;
        next = c->arena_free.erase(next);
    }
    if (next != c->arena_free.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += len;
            return;
        }
    }
    c->arena_free[off] = len;
}

template <class T>
int dalloc(gmp_ctx* c, T** p, size_t n) {
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    if (c->budget && c->used + bytes > c->budget)
        return fail(c, GMP_ERR_OOM, "memory budget exceeded: %zu + %zu > %llu bytes", (size_t)c->used, bytes,
                    (unsigned long long)c->budget);
    void* q = nullptr;
    if (c->arena) {
        q = arena_take(c, bytes);
        if (!q) return fail(c, GMP_ERR_OOM, "bound workspace exhausted: no free run of %zu bytes", bytes);
    } else {
        cudaError_t e = c->stream_alloc ? cudaMallocAsync(&q, bytes, c->stream) : cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, GMP_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    *p = static_cast<T*>(q);
    c->used += bytes;
    c->sizes[q] = bytes;
    return GMP_OK;
}

template <class T>
void dfree(gmp_ctx* c, T** p) {
    if (*p) {
        auto it = c->sizes.find((void*)*p);
        if (it != c->sizes.end()) {
            c->used -= it->second;
            c->sizes.erase(it);
        }
        if (c->arena_blocks.count((void*)*p)) arena_give(c, (void*)*p);
        else if (c->stream_alloc) cudaFreeAsync((void*)*p, c->stream);
        else cudaFree((void*)*p);
        *p = nullptr;
    }
}

// (Re)allocate a workspace buffer only when it must grow.
template <class T>
int ensure(gmp_ctx* c, T** p, size_t n) {
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    if (*p) {
        auto it = c->sizes.find((void*)*p);
        if (it != c->sizes.end() && it->second >= bytes) return GMP_OK;
        dfree(c, p);
    }
    return dalloc(c, p, n);
}

template <class T>
int upload(gmp_ctx* c, T* d, const T* h, size_t n) {
    if (n == 0) return GMP_OK;
    GMP_CUDA(c, cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return GMP_OK;
}

void drop_graph(Batch& b) {
    for (auto& kv : b.execs) cudaGraphExecDestroy(kv.second);
    b.execs.clear();
    b.exec = nullptr;
    b.key = BatchKey{};
}

void drop_events(Batch& b) {
    for (cudaEvent_t e : b.ev) cudaEventDestroy(e);
    b.ev.clear();
}

void free_batch(gmp_ctx* c) {
    Batch& b = c->b;
    drop_graph(b);
    drop_events(b);
    if (b.done) {
        cudaEventDestroy(b.done);
        b.done = nullptr;
    }
    dfree(c, &b.dq);
    dfree(c, &b.prefix);
    dfree(c, &b.tau);
    dfree(c, &b.th);
    dfree(c, &b.tflag);
    dfree(c, &b.list_e);
    dfree(c, &b.list_tau);
    dfree(c, &b.dep);
    dfree(c, &b.qs);
    dfree(c, &b.routes);
    dfree(c, &b.ant_steps);
    dfree(c, &b.ant_wait);
    dfree(c, &b.best_route);
    dfree(c, &b.route_out);
    dfree(c, &b.tickets);
    dfree(c, &b.ant_log);
    dfree(c, &b.tabu);
    dfree(c, &b.res);
    dfree(c, &b.ctr);
    dfree(c, &b.qstate);
    dfree(c, &b.qflag);
    dfree(c, &b.misc);
    dfree(c, &b.hdist);
    dfree(c, &b.hqueue);
    dfree(c, &b.hstamp);
    dfree(c, &b.tail_list);
    dfree(c, &b.tail_state);
    dfree(c, &b.tail_tabu);
    b.staged = b.ran = false;
}

// Forget (without freeing) what a view borrowed.
void drop_borrowed(gmp_ctx* c) {
    if (c->lender) {
        c->row_ptr = c->col = c->len = c->in_ptr = c->in_edge = c->in_tail = c->ff = c->cap = nullptr;
        c->speed = nullptr;
        c->lanes = c->lanes_in = nullptr;
        c->x = c->y = nullptr;
        c->nph = c->ephase = nullptr;
        c->cycle = c->offset = c->green = nullptr;
    }
    if (!c->own_state) {
        c->order = nullptr;
        c->red = c->veh = c->tick_leave = nullptr;
        c->rec = nullptr;
        c->tick_K = nullptr;
    }
    if (c->lender) --c->lender->views;
    if (c->state_lender) --c->state_lender->views;
    c->lender = c->state_lender = nullptr;
    c->own_state = true;
}

void free_graph(gmp_ctx* c) {
    free_batch(c);
    drop_borrowed(c);
    dfree(c, &c->row_ptr);
    dfree(c, &c->col);
    dfree(c, &c->len);
    dfree(c, &c->in_ptr);
    dfree(c, &c->in_edge);
    dfree(c, &c->in_tail);
    dfree(c, &c->ff);
    dfree(c, &c->cap);
    dfree(c, &c->speed);
    dfree(c, &c->lanes);
    dfree(c, &c->lanes_in);
    dfree(c, &c->x);
    dfree(c, &c->y);
    dfree(c, &c->nph);
    dfree(c, &c->ephase);
    dfree(c, &c->order);
    dfree(c, &c->cycle);
    dfree(c, &c->offset);
    dfree(c, &c->green);
    dfree(c, &c->red);
    dfree(c, &c->veh);
    dfree(c, &c->rec);
    dfree(c, &c->tick_leave);
    dfree(c, &c->tick_K);
    c->has_graph = false;
    c->N = c->E = 0;
    c->hin_edge.reset();
    c->red_high = false;
}

uint32_t hsat_of(const gmp_ctx* c) { return c->prm.h_sat_ms ? c->prm.h_sat_ms : kHsatDefault; }

// What the intersection passes read and write, on this context's graph and traffic state.
QueueTables queue_tables(const gmp_ctx* c) {
    QueueTables t{};
    t.n_nodes = c->N;
    t.h_sat = hsat_of(c);
    t.thr = c->prm.thr_permille;
    t.row_ptr = c->row_ptr;
    t.in_ptr = c->in_ptr;
    t.in_edge = c->in_edge;
    t.in_tail = c->in_tail;
    t.nph = c->nph;
    t.cycle = c->cycle;
    t.offset = c->offset;
    t.green = c->green;
    t.ephase = c->ephase;
    t.lanes = c->lanes_in;
    t.cap = c->cap;
    t.ff = c->ff;
    t.veh = c->veh;
    t.red = c->red;
    t.order = c->order;
    t.rec = c->rec;
    t.leave = c->tick_leave;
    t.K = c->tick_K;
    return t;
}

// Densities or signals or params changed: rebuild the phase orders and every road record.
int refresh_dynamic(gmp_ctx* c) {
    GMP_CUDA(c, launch_queue(c->stream, queue_tables(c), c->max_phases, QueuePass::kRefresh));
    return GMP_OK;
}

int sync(gmp_ctx* c) {
    GMP_CUDA(c, cudaStreamSynchronize(c->stream));
    return GMP_OK;
}

// Copy src's traffic state (vehicles, red times, phase order, road records) into dst's own arrays, on
// dst's stream. Both contexts share one static graph.
int copy_state(gmp_ctx* dst, const gmp_ctx* src) {
    cudaStream_t s = dst->stream;
    GMP_CUDA(dst, cudaMemcpyAsync(dst->veh, src->veh, std::max<size_t>(dst->E, 1) * 4, cudaMemcpyDeviceToDevice, s));
    GMP_CUDA(dst, cudaMemcpyAsync(dst->red, src->red, (size_t)dst->N * kMaxPhases * 4, cudaMemcpyDeviceToDevice, s));
    GMP_CUDA(dst, cudaMemcpyAsync(dst->order, src->order, (size_t)dst->N * kMaxPhases, cudaMemcpyDeviceToDevice, s));
    GMP_CUDA(dst, cudaMemcpyAsync(dst->rec, src->rec, std::max<size_t>(dst->E, 1) * sizeof(EdgeRec),
                                  cudaMemcpyDeviceToDevice, s));
    dst->red_high = src->red_high;
    return GMP_OK;
}

uint32_t tflag_words(const gmp_ctx* c) { return (c->E + 31u) / 32u; }

// The pheromone layout of the next job (results are the same in both).
bool use_sparse(const gmp_ctx* c) {
    if (c->prm.mode == GMP_MODE_PERSISTENT || (c->prm.flags & GMP_FLAG_RANDOM_TAU)) return false;
    if (c->prm.tau_layout == GMP_TAU_SPARSE) return true;
    if (c->prm.tau_layout == GMP_TAU_DENSE) return false;
    return c->E >= kSparseMinEdges;
}

// Moves per ant, forward and back: min(2(N - 1), 4096) unless set, the length of a complete
// depth-first walk over the graph.
uint32_t default_max_steps(const gmp_ctx* c) {
    if (c->prm.max_steps) return c->prm.max_steps;
    const uint64_t n2 = c->N > 0 ? 2ull * (c->N - 1u) : 0ull;
    return n2 < 4096u ? (uint32_t)n2 : 4096u;
}

int pick_lanes(const gmp_ctx* c) {
    if (c->prm.lanes_per_ant) return (int)c->prm.lanes_per_ant;
    return (int)default_lanes(c->maxdeg);
}

int check_query(gmp_ctx* c, const gmp_query& q, uint32_t idx) {
    if (q.src >= c->N || q.dst >= c->N)
        return fail(c, GMP_ERR_INVALID_ARG, "query %u: node out of range (src %u, dst %u, N %u)", idx, q.src, q.dst, c->N);
    if (q.n_ants == 0 || q.n_iter == 0) return fail(c, GMP_ERR_INVALID_ARG, "query %u: n_ants and n_iter must be >= 1", idx);
    if ((uint64_t)q.n_ants * q.n_iter > 0xFFFFFFFFull)
        return fail(c, GMP_ERR_INVALID_ARG, "query %u: n_ants * n_iter must be < 2^32", idx);
    if (!(q.alpha >= 0.0f && q.alpha <= 8.0f && q.beta >= 0.0f && q.beta <= 8.0f))
        return fail(c, GMP_ERR_UNSUPPORTED, "query %u: alpha and beta must lie in [0, 8]", idx);
    if (!(q.rho >= 0.0f && q.rho < 1.0f)) return fail(c, GMP_ERR_INVALID_ARG, "query %u: rho must lie in [0, 1)", idx);
    return GMP_OK;
}

// Exponents as the kernels take them: integers as integers (repeated multiplication); otherwise both
// as binary32 bits with kQueryFracExp set in `active` (the 2^L score). Call after `active` is set.
void set_exponents(DevQuery& d, float alpha, float beta) {
    if (floorf(alpha) != alpha || floorf(beta) != beta) {
        memcpy(&d.alpha, &alpha, sizeof alpha);
        memcpy(&d.beta, &beta, sizeof beta);
        if (d.active) d.active |= kQueryFracExp;
    } else {
        d.alpha = (uint32_t)alpha;
        d.beta = (uint32_t)beta;
    }
}

int record(gmp_ctx* c, Batch& b, size_t i) {
    GMP_CUDA(c, cudaEventRecordWithFlags(b.ev[i], c->stream, cudaEventRecordExternal));
    return GMP_OK;
}

ConstructArgs construct_args(gmp_ctx* c);

// Arguments of the iteration-end kernel for a job's workspace (the context supplies the queue state).
IterEndArgs iter_end_args(gmp_ctx* c, uint32_t Q, const DevQuery* dq, uint64_t* tau, uint2* th,
                          unsigned long long* dep, QueryState* qs, const uint32_t* routes, const uint32_t* ant_steps,
                          const uint32_t* ant_wait, uint32_t* best_route, uint32_t max_steps) {
    IterEndArgs e{};
    e.n_queries = Q;
    e.n_edges = c->E;
    e.n_nodes = c->N;
    e.max_steps = max_steps;
    e.flags = c->prm.flags;
    e.q = dq;
    e.tau = tau;
    e.th = th;
    e.dep = dep;
    e.qs = qs;
    e.routes = routes;
    e.ant_steps = ant_steps;
    e.ant_wait = ant_wait;
    e.best_route = best_route;
    e.qt = queue_tables(c);
    return e;
}

// Exact Calc_Dist of every colony of the job, ahead of the initialisation that reads it.
int enqueue_exact_h(gmp_ctx* c) {
    Batch& b = c->b;
    if (!b.exact_h) return GMP_OK;
    GMP_CUDA(c, cudaMemsetAsync(b.misc + 2, 0, 4, c->stream));
    GMP_CUDA(c, launch_exact_h(c->stream, b.Q, c->N, b.dq, c->in_ptr, c->in_edge, c->in_tail, c->rec, c->h_delta,
                               c->prm.level_limit,
                               b.hdist, b.hqueue, b.hstamp, b.misc + 2));
    return GMP_OK;
}

// The persistent job: init, one persistent launch, result rows.
int enqueue_persistent(gmp_ctx* c) {
    Batch& b = c->b;
    cudaStream_t s = c->stream;
    const bool timed = b.timed;
    if (timed) GMP_TRY(record(c, b, 0));
    GMP_TRY(enqueue_exact_h(c));
    GMP_CUDA(c, launch_init_batch(s, b.Q, c->E, b.dq, c->col, c->x, c->y, c->kappa, c->prm.flags, b.tau, b.th,
                                  b.dep, b.qs, b.tickets, b.maxI, 0u, nullptr, 0u, b.exact_h ? b.hdist : nullptr, c->N,
                                  true));
    GMP_CUDA(c, launch_persistent_init(s, b.Q, b.maxI, b.dq, b.ctr, b.qstate, b.qflag, b.misc));
    if (b.tabu && b.tabu_used) GMP_CUDA(c, cudaMemsetAsync(b.tabu, 0, b.tabu_used * 4, s));
    if (timed) GMP_TRY(record(c, b, 1));
    PersistentArgs p{};
    p.c = construct_args(c);
    p.ctr = b.ctr;
    p.qstate = b.qstate;
    p.qflag = b.qflag;
    p.misc = b.misc;
    p.tau = b.tau;
    p.th = b.th;
    p.best_route = b.best_route;
    p.qt = queue_tables(c);
    p.n_nodes = c->N;
    p.max_iter = b.maxI;
    p.flags = c->prm.flags;
    p.node_chunk = c->prm.queue_chunk ? c->prm.queue_chunk : 16u;
    p.spin_limit = c->prm.poll_limit ? c->prm.poll_limit : 1u << 23;  // idle polls (~0.3 us each) before a timeout
    GMP_CUDA(c, launch_persistent(s, b.kc, p));
    if (timed) GMP_TRY(record(c, b, 2));
    GMP_CUDA(c, launch_finalize(s, b.Q, b.dq, b.qs, b.best_route, c->col, b.max_steps, b.res, b.route_out));
    if (timed) GMP_TRY(record(c, b, 3));
    b.launches = b.exact_h ? 5 : 4;
    return GMP_OK;
}

ConstructArgs construct_args(gmp_ctx* c) {
    Batch& b = c->b;
    ConstructArgs a{};
    a.rec = c->rec;
    a.row_ptr = c->row_ptr;
    a.col = c->col;
    a.queries = b.dq;
    a.ant_prefix = b.prefix;
    a.tau = b.tau;
    a.th = b.th;
    a.dep = b.dep;
    a.qs = b.qs;
    a.routes = b.routes;
    a.rwait = b.routes + (size_t)b.total_ants * b.max_steps;
    a.ant_steps = b.ant_steps;
    a.ant_wait = b.ant_wait;
    a.ant_log = b.log_entries ? b.ant_log : nullptr;  // sized at staging
    a.tickets = b.tickets;
    a.tabu_global = b.tabu;
    a.n_queries = b.Q;
    a.total_ants = b.total_ants;
    a.n_edges = c->E;
    a.max_steps = b.max_steps;
    a.tabu_words = (c->N + 31u) / 32u;
    a.t_dep = c->prm.t_dep_ms;
    a.thr_on = c->prm.thr_permille != kThrOff;
    a.tabu_in_smem = b.kc.tabu_in_smem ? 1u : 0u;
    a.kappa = c->kappa;
    a.sparse = b.sparse ? 1u : 0u;
    a.tflag_words = tflag_words(c);
    a.tflag = b.tflag;
    a.list_e = b.list_e;
    a.list_tau = b.list_tau;
    a.handoff_moves = b.handoff;
    a.tail_list = b.tail_list;
    a.tail_state = b.tail_state;
    a.tail_tabu = b.tail_tabu;
    return a;
}

// Issue the whole job on the stream (inside a capture or directly).
// Per-kernel timing events of the iterative job: [0] start, [1] after init, [2] after the chains join,
// [3] after the result rows; then per chain its start and, per iteration, after construction and after
// the iteration end.
size_t branch_event_base(const Batch& b, size_t j) {
    size_t base = 4;
    for (size_t i = 0; i < j; ++i) base += 1 + 2 * (size_t)b.br[i].maxI;
    return base;
}

size_t job_event_count(const Batch& b) {
    if (b.persistent) return 4;
    return branch_event_base(b, b.br.size());
}

int ensure_branch_streams(gmp_ctx* c, size_t n) {
    if (!c->bfork) GMP_CUDA(c, cudaEventCreateWithFlags(&c->bfork, cudaEventDisableTiming));
    while (c->bstreams.size() < n) {
        cudaStream_t st = nullptr;
        GMP_CUDA(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        c->bstreams.push_back(st);
        cudaEvent_t e = nullptr;
        GMP_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->bjoin.push_back(e);
    }
    return GMP_OK;
}

// Issue the whole job on the stream (inside a capture or directly). Colony ranges run as concurrent
// chains (fork from the context's stream after init, join before the result rows): a chain moves on to
// its next iteration as soon as its own colonies finish, so the job takes as long as its slowest chain
// instead of the sum over iterations of the slowest ant of any colony.
int enqueue_job(gmp_ctx* c) {
    Batch& b = c->b;
    if (b.persistent) return enqueue_persistent(c);
    cudaStream_t s = c->stream;
    const bool timed = b.timed;
    const size_t B = b.br.size();
    uint64_t n = 0;
    if (timed) GMP_TRY(record(c, b, 0));
    GMP_TRY(enqueue_exact_h(c));
    if (b.exact_h) ++n;
    GMP_CUDA(c, launch_init_batch(s, b.Q, c->E, b.dq, c->col, c->x, c->y, c->kappa, c->prm.flags, b.tau, b.th,
                                  b.dep, b.qs, b.tickets, b.maxI * (uint32_t)B * (b.handoff ? 3u : 1u),
                                  b.sparse ? 1u : 0u, b.tflag,
                                  tflag_words(c), b.exact_h ? b.hdist : nullptr, c->N, false));
    ++n;
    if (timed) GMP_TRY(record(c, b, 1));
    // global visited bitmaps start clean; each walk clears its own bits when it ends
    if (b.tabu && b.tabu_used) GMP_CUDA(c, cudaMemsetAsync(b.tabu, 0, b.tabu_used * 4, s));
    if (B > 1) {
        GMP_TRY(ensure_branch_streams(c, B));
        GMP_CUDA(c, cudaEventRecord(c->bfork, s));
    }
    const ConstructArgs base = construct_args(c);
    for (size_t j = 0; j < B; ++j) {
        const Batch::Branch& r = b.br[j];
        cudaStream_t bs = B > 1 ? c->bstreams[j] : s;
        if (B > 1) GMP_CUDA(c, cudaStreamWaitEvent(bs, c->bfork, 0));
        const size_t eb = branch_event_base(b, j);
        if (timed) GMP_CUDA(c, cudaEventRecordWithFlags(b.ev[eb], bs, cudaEventRecordExternal));
        ConstructArgs a = base;
        const size_t co = (size_t)r.q0 * c->E;
        a.queries = b.dq + r.q0;
        a.ant_prefix = b.prefix + r.q0;
        a.tau = b.tau + co;
        a.th = b.th + co;
        a.dep = b.dep + co;
        a.qs = b.qs + r.q0;
        a.tickets = b.tickets + (size_t)j * b.maxI;
        if (b.handoff) {  // the tail counters follow the tickets: B * maxI suspended, then B * maxI taken up
            a.tail_count = b.tickets + ((size_t)B + j) * b.maxI;
            a.tail_claim = b.tickets + (2 * (size_t)B + j) * b.maxI;
        }
        if (b.sparse) {
            a.tflag = b.tflag + (size_t)r.q0 * a.tflag_words;
            a.list_e = b.list_e + co;
            a.list_tau = b.list_tau + co;
        }
        a.tabu_global = b.tabu ? b.tabu + r.tabu_off : nullptr;
        a.n_queries = r.q1 - r.q0;
        a.total_ants = r.ants;
        a.ticket_base = r.ticket_base;
        a.tabu_in_smem = r.kc.tabu_in_smem ? 1u : 0u;
        IterEndArgs e = iter_end_args(c, r.q1 - r.q0, b.dq + r.q0, b.tau + co, b.th + co, b.dep + co, b.qs + r.q0,
                                      b.routes, b.ant_steps, b.ant_wait, b.best_route + (size_t)r.q0 * b.max_steps,
                                      b.max_steps);
        const uint32_t n_nodes = e.n_nodes;
        if (b.sparse) {
            e.sparse = 1;
            e.list_e = b.list_e + co;
            e.list_tau = b.list_tau + co;
        }
        for (uint32_t it = 0; it < r.maxI; ++it) {
            GMP_CUDA(c, launch_construct(bs, r.kc, a, it));
            if (b.handoff) {  // the walks the construction launch suspended
                GMP_CUDA(c, launch_construct_tail(bs, r.kc_tail, a, it));
                ++n;
            }
            if (timed) GMP_CUDA(c, cudaEventRecordWithFlags(b.ev[eb + 1 + 2 * it], bs, cudaEventRecordExternal));
            e.it = it;
            // the queue update of iteration `it` runs once, in chain it mod B (densities are fixed during a
            // job, so every chain would compute the same order): the chains share that work evenly
            e.n_nodes = (it % B == j) ? n_nodes : 0u;
            GMP_CUDA(c, launch_iter_end(bs, e));
            if (e.n_nodes && b.queue_general) {  // the iteration end updated the intersections with <= 2 phases
                GMP_CUDA(c, launch_queue_general(bs, e.qt, QueuePass::kIterate));
                ++n;
            }
            if (timed) GMP_CUDA(c, cudaEventRecordWithFlags(b.ev[eb + 2 + 2 * it], bs, cudaEventRecordExternal));
            n += 2;
        }
        if (B > 1) {
            GMP_CUDA(c, cudaEventRecord(c->bjoin[j], bs));
            GMP_CUDA(c, cudaStreamWaitEvent(s, c->bjoin[j], 0));
        }
    }
    if (timed) GMP_TRY(record(c, b, 2));
    GMP_CUDA(c, launch_finalize(s, b.Q, b.dq, b.qs, b.best_route, c->col, b.max_steps, b.res, b.route_out));
    ++n;
    if (timed) GMP_TRY(record(c, b, 3));
    b.launches = n;
    return GMP_OK;
}

BatchKey key_of(const gmp_ctx* c) {
    const Batch& b = c->b;
    BatchKey k{};
    k.Q = b.Q;
    k.chunk = c->prm.queue_chunk;
    k.poll_limit = c->prm.poll_limit;
    k.level_limit = c->prm.level_limit;
    k.branches = (uint32_t)b.br.size();
    k.sparse = b.sparse ? 1u : 0u;
    k.maxI = b.maxI;
    k.total_ants = b.total_ants;
    k.max_steps = b.max_steps;
    k.flags = c->prm.flags;
    k.lanes = (uint32_t)(b.kc.lanes * 16 + b.kc.slots) | (b.kc.lockstep ? 0x10000u : 0u) |
              (b.persistent ? 0x20000u : 0u);
    k.grid = (uint32_t)b.kc.grid;
    k.thr_on = c->prm.thr_permille != kThrOff;
    k.t_dep = c->prm.t_dep_ms;
    k.log_entries = b.log_entries;
    k.handoff = b.handoff;
    k.ptrs[0] = b.tau;
    k.ptrs[1] = b.routes;
    k.ptrs[2] = b.tabu;
    k.ptrs[3] = c->rec;
    k.ptrs[4] = b.th;
    k.ptrs[5] = b.dep;
    return k;
}

}  // namespace

// =====================================================================================================
extern "C" {

const char* gmp_strerror(int code) {
    switch (code) {
        case GMP_OK: return "ok";
        case GMP_ERR_INVALID_ARG: return "invalid argument";
        case GMP_ERR_NO_ROUTE: return "no route found";
        case GMP_ERR_OOM: return "out of device memory or memory budget";
        case GMP_ERR_CUDA: return "CUDA error";
        case GMP_ERR_TIMEOUT: return "device wait timed out";
        case GMP_ERR_UNSUPPORTED: return "unsupported";
        case GMP_ERR_BUFFER: return "buffer too small";
        case GMP_ERR_STATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* gmp_last_error(const gmp_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int gmp_create(gmp_ctx** out, int device, uint64_t mem_budget_bytes, void* cuda_stream) {
    if (!out) return GMP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return GMP_ERR_CUDA;
    }
    if (device < 0 || device >= n) return GMP_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return GMP_ERR_CUDA;
    gmp_ctx* c = new gmp_ctx();
    c->device = device;
    c->budget = mem_budget_bytes;
    c->prm.thr_permille = GMP_THRESHOLD_OFF;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return GMP_ERR_CUDA;
    }
    c->stream = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
    *out = c;
    return GMP_OK;
}

void gmp_destroy(gmp_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_graph(c);
    for (cudaStream_t st : c->bstreams) cudaStreamDestroy(st);
    for (cudaEvent_t e : c->bjoin) cudaEventDestroy(e);
    if (c->bfork) cudaEventDestroy(c->bfork);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

int gmp_set_stream(gmp_ctx* c, void* cuda_stream) {
    if (!c) return GMP_ERR_INVALID_ARG;
    c->stream = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
    return GMP_OK;
}

int gmp_bind_workspace(gmp_ctx* c, void* dev_ptr, uint64_t bytes) {
    if (!c) return GMP_ERR_INVALID_ARG;
    if (c->has_graph || !c->sizes.empty())
        return fail(c, GMP_ERR_STATE, "bind the workspace before gmp_load_graph (the context holds device memory)");
    if (!dev_ptr) {
        c->arena = nullptr;
        c->arena_bytes = 0;
        c->arena_free.clear();
        c->arena_blocks.clear();
        return GMP_OK;
    }
    if ((uintptr_t)dev_ptr % 256u != 0 || bytes < 256u)
        return fail(c, GMP_ERR_INVALID_ARG, "workspace must be 256-byte aligned and at least 256 bytes");
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, dev_ptr) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
        attr.device != c->device) {
        cudaGetLastError();
        return fail(c, GMP_ERR_INVALID_ARG, "workspace must be device memory of the context's GPU");
    }
    c->arena = static_cast<char*>(dev_ptr);
    c->arena_bytes = bytes & ~(uint64_t)255u;
    c->arena_free.clear();
    c->arena_blocks.clear();
    c->arena_free[0] = c->arena_bytes;
    return GMP_OK;
}

int gmp_load_graph(gmp_ctx* c, uint32_t N, uint32_t E, const uint32_t* row_ptr, const uint32_t* col,
                   const uint32_t* length_dm, const uint16_t* speed_kmh, const uint8_t* lanes, const int32_t* x_dm,
                   const int32_t* y_dm) {
    if (!c) return GMP_ERR_INVALID_ARG;
    if (N == 0 || N >= (1u << 31) || E >= (1u << 31))
        return fail(c, GMP_ERR_INVALID_ARG, "need 1 <= N < 2^31 and E < 2^31");
    if (!row_ptr || !x_dm || !y_dm || (E && (!col || !length_dm || !speed_kmh || !lanes)))
        return fail(c, GMP_ERR_INVALID_ARG, "null array");
    if (row_ptr[0] != 0 || row_ptr[N] != E) return fail(c, GMP_ERR_INVALID_ARG, "row_ptr must start at 0 and end at E");
    uint32_t maxdeg = 0;
    for (uint32_t v = 0; v < N; ++v) {
        if (row_ptr[v + 1] < row_ptr[v]) return fail(c, GMP_ERR_INVALID_ARG, "row_ptr not monotone at %u", v);
        maxdeg = std::max(maxdeg, row_ptr[v + 1] - row_ptr[v]);
        if (x_dm[v] > kCoordLimit || x_dm[v] < -kCoordLimit || y_dm[v] > kCoordLimit || y_dm[v] < -kCoordLimit)
            return fail(c, GMP_ERR_INVALID_ARG, "coordinate of node %u beyond +-2^27 dm", v);
    }
    uint32_t vmax = 1;
    std::vector<uint32_t> in_ptr(N + 1, 0), in_edge(E), in_tail(E);
    for (uint32_t e = 0; e < E; ++e) {
        if (col[e] >= N) return fail(c, GMP_ERR_INVALID_ARG, "col[%u] out of range", e);
        if (length_dm[e] == 0 || speed_kmh[e] == 0 || lanes[e] == 0)
            return fail(c, GMP_ERR_INVALID_ARG, "road %u: length, speed and lanes must be >= 1", e);
        vmax = std::max<uint32_t>(vmax, speed_kmh[e]);
        in_ptr[col[e] + 1]++;
    }
    for (uint32_t v = 0; v < N; ++v) in_ptr[v + 1] += in_ptr[v];
    {
        std::vector<uint32_t> fill(in_ptr.begin(), in_ptr.end() - 1), tail_of(E);
        for (uint32_t e = 0; e < E; ++e) in_edge[fill[col[e]]++] = e;
        for (uint32_t u = 0; u < N; ++u)
            for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tail_of[e] = u;
        for (uint32_t i = 0; i < E; ++i) in_tail[i] = tail_of[in_edge[i]];
    }
    if (c->views) return fail(c, GMP_ERR_STATE, "other contexts view this context's graph");
    cudaSetDevice(c->device);
    sync(c);
    free_graph(c);
    c->N = N;
    c->E = E;
    c->maxdeg = maxdeg;
    c->self_loops = false;
    for (uint32_t v = 0; v < N && !c->self_loops; ++v)
        for (uint32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) c->self_loops = c->self_loops || col[e] == v;
    c->hx.assign(x_dm, x_dm + N);
    c->hy.assign(y_dm, y_dm + N);
    c->kappa = (uint32_t)((360ull << 16) / vmax);
    c->max_phases = 0;  // no signals until gmp_set_signals
    {
        uint64_t ff_sum = 0;  // free-flow times as the road kernels compute them (a tuning input only)
        for (uint32_t e = 0; e < E; ++e) ff_sum += ((uint64_t)length_dm[e] * 360u + speed_kmh[e] / 2u) / speed_kmh[e];
        c->h_delta = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(16u * (E ? ff_sum / E : 1u), 1u), 1u << 27);
    }
    GMP_TRY(dalloc(c, &c->row_ptr, N + 1));
    GMP_TRY(dalloc(c, &c->col, E));
    GMP_TRY(dalloc(c, &c->len, E));
    GMP_TRY(dalloc(c, &c->in_ptr, N + 1));
    GMP_TRY(dalloc(c, &c->in_edge, E));
    GMP_TRY(dalloc(c, &c->in_tail, E));
    GMP_TRY(dalloc(c, &c->ff, E));
    GMP_TRY(dalloc(c, &c->cap, E));
    GMP_TRY(dalloc(c, &c->speed, E));
    GMP_TRY(dalloc(c, &c->lanes, E));
    GMP_TRY(dalloc(c, &c->lanes_in, E));
    GMP_TRY(dalloc(c, &c->x, N));
    GMP_TRY(dalloc(c, &c->y, N));
    GMP_TRY(dalloc(c, &c->nph, N));
    GMP_TRY(dalloc(c, &c->ephase, E));
    GMP_TRY(dalloc(c, &c->order, (size_t)N * kMaxPhases));
    GMP_TRY(dalloc(c, &c->cycle, N));
    GMP_TRY(dalloc(c, &c->offset, N));
    GMP_TRY(dalloc(c, &c->green, (size_t)N * kMaxPhases));
    GMP_TRY(dalloc(c, &c->red, (size_t)N * kMaxPhases));
    GMP_TRY(dalloc(c, &c->veh, E));
    GMP_TRY(dalloc(c, &c->rec, E));
    GMP_TRY(dalloc(c, &c->tick_leave, E));
    GMP_TRY(dalloc(c, &c->tick_K, N));
    GMP_TRY(upload(c, c->row_ptr, row_ptr, N + 1));
    GMP_TRY(upload(c, c->col, col, E));
    GMP_TRY(upload(c, c->len, length_dm, E));
    GMP_TRY(upload(c, c->speed, speed_kmh, E));
    GMP_TRY(upload(c, c->lanes, lanes, E));
    GMP_TRY(upload(c, c->x, x_dm, N));
    GMP_TRY(upload(c, c->y, y_dm, N));
    GMP_TRY(upload(c, c->in_ptr, in_ptr.data(), N + 1));
    GMP_TRY(upload(c, c->in_edge, in_edge.data(), E));
    GMP_TRY(upload(c, c->in_tail, in_tail.data(), E));
    GMP_CUDA(c, cudaMemsetAsync(c->nph, 0, N, c->stream));
    GMP_CUDA(c, cudaMemsetAsync(c->ephase, 0, std::max<size_t>(E, 1), c->stream));
    GMP_CUDA(c, cudaMemsetAsync(c->cycle, 0, N * 4ull, c->stream));
    GMP_CUDA(c, cudaMemsetAsync(c->offset, 0, N * 4ull, c->stream));
    GMP_CUDA(c, cudaMemsetAsync(c->green, 0, N * 4ull * kMaxPhases, c->stream));
    GMP_CUDA(c, cudaMemsetAsync(c->red, 0, N * 4ull * kMaxPhases, c->stream));
    GMP_CUDA(c, cudaMemsetAsync(c->veh, 0, std::max<size_t>(E, 1) * 4, c->stream));
    GMP_CUDA(c, launch_edge_static(c->stream, E, c->in_edge, c->len, c->speed, c->lanes, c->ff, c->cap, c->lanes_in));
    GMP_TRY(refresh_dynamic(c));
    GMP_TRY(sync(c));
    c->hin_edge = std::make_shared<const std::vector<uint32_t>>(std::move(in_edge));
    c->red_high = false;
    c->has_graph = true;
    return GMP_OK;
}

int gmp_share_graph(gmp_ctx* c, gmp_ctx* owner, int own_state) {
    if (!c || !owner || c == owner) return GMP_ERR_INVALID_ARG;
    if (!owner->has_graph) return fail(c, GMP_ERR_STATE, "the owner holds no graph");
    if (owner->device != c->device) return fail(c, GMP_ERR_INVALID_ARG, "both contexts must be on one device");
    if (c->views) return fail(c, GMP_ERR_STATE, "other contexts view this context's graph");
    cudaSetDevice(c->device);
    sync(c);
    free_graph(c);
    gmp_ctx* root = owner->lender ? owner->lender : owner;
    c->N = owner->N;
    c->E = owner->E;
    c->maxdeg = owner->maxdeg;
    c->self_loops = owner->self_loops;
    c->kappa = owner->kappa;
    c->h_delta = owner->h_delta;
    c->max_phases = owner->max_phases;
    c->hx = owner->hx;
    c->hy = owner->hy;
    c->row_ptr = owner->row_ptr;
    c->col = owner->col;
    c->len = owner->len;
    c->in_ptr = owner->in_ptr;
    c->in_edge = owner->in_edge;
    c->in_tail = owner->in_tail;
    c->ff = owner->ff;
    c->cap = owner->cap;
    c->speed = owner->speed;
    c->lanes = owner->lanes;
    c->lanes_in = owner->lanes_in;
    c->hin_edge = owner->hin_edge;
    c->x = owner->x;
    c->y = owner->y;
    c->nph = owner->nph;
    c->ephase = owner->ephase;
    c->cycle = owner->cycle;
    c->offset = owner->offset;
    c->green = owner->green;
    c->lender = root;
    ++root->views;
    c->prm.thr_permille = owner->prm.thr_permille;
    c->prm.h_sat_ms = owner->prm.h_sat_ms;
    if (own_state) {  // a copy of the owner's traffic state, ordered after the owner's queued work
        c->own_state = true;
        GMP_TRY(dalloc(c, &c->order, (size_t)c->N * kMaxPhases));
        GMP_TRY(dalloc(c, &c->red, (size_t)c->N * kMaxPhases));
        GMP_TRY(dalloc(c, &c->veh, c->E));
        GMP_TRY(dalloc(c, &c->rec, c->E));
        GMP_TRY(dalloc(c, &c->tick_leave, c->E));
        GMP_TRY(dalloc(c, &c->tick_K, c->N));
        GMP_CUDA(c, cudaStreamSynchronize(owner->stream));
        GMP_TRY(copy_state(c, owner));
        GMP_TRY(sync(c));
    } else {
        c->own_state = false;
        c->state_lender = owner;
        ++owner->views;
        c->order = owner->order;
        c->red = owner->red;
        c->veh = owner->veh;
        c->rec = owner->rec;
        c->tick_leave = owner->tick_leave;
        c->tick_K = owner->tick_K;
    }
    c->has_graph = true;
    return GMP_OK;
}

int gmp_set_signals(gmp_ctx* c, const uint8_t* n_phases, const uint32_t* cycle_ms, const uint32_t* offset_ms,
                    const uint32_t* green_ms, const uint8_t* edge_phase) {
    if (!c) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (!n_phases || !cycle_ms || !offset_ms || !green_ms || (c->E && !edge_phase))
        return fail(c, GMP_ERR_INVALID_ARG, "null array");
    if (c->lender || c->views) return fail(c, GMP_ERR_STATE, "signal programmes of a shared graph are fixed");
    std::vector<uint32_t> row(c->N + 1);
    for (uint32_t v = 0; v < c->N; ++v) {
        const uint32_t P = n_phases[v];
        if (P > kMaxPhases) return fail(c, GMP_ERR_UNSUPPORTED, "node %u: more than 8 phases", v);
        if (P == 0) continue;
        const uint32_t cy = cycle_ms[v];
        if (cy == 0 || cy > kCycleMask) return fail(c, GMP_ERR_INVALID_ARG, "node %u: cycle must be in 1..2^24-1 ms", v);
        if (offset_ms[v] >= cy) return fail(c, GMP_ERR_INVALID_ARG, "node %u: offset must be below the cycle", v);
        uint64_t sum = 0;
        for (uint32_t p = 0; p < P; ++p) {
            if (green_ms[(size_t)v * kMaxPhases + p] == 0)
                return fail(c, GMP_ERR_INVALID_ARG, "node %u: every phase needs green time", v);
            sum += green_ms[(size_t)v * kMaxPhases + p];
        }
        if (sum != cy) return fail(c, GMP_ERR_INVALID_ARG, "node %u: green times must add up to the cycle", v);
    }
    std::vector<uint32_t> hcol(c->E);
    cudaSetDevice(c->device);
    if (c->E) GMP_CUDA(c, cudaMemcpy(hcol.data(), c->col, c->E * 4ull, cudaMemcpyDeviceToHost));
    for (uint32_t e = 0; e < c->E; ++e) {
        const uint32_t P = n_phases[hcol[e]];
        if (P > 0 && edge_phase[e] >= P)
            return fail(c, GMP_ERR_INVALID_ARG, "road %u: approach phase %u beyond the head's %u phases", e, edge_phase[e], P);
    }
    sync(c);
    // phase-major greens, approach phases in slot order (host staging, waited for below)
    std::vector<uint32_t> planes((size_t)c->N * kMaxPhases);
    for (uint32_t v = 0; v < c->N; ++v)
        for (uint32_t p = 0; p < kMaxPhases; ++p) planes[(size_t)p * c->N + v] = green_ms[(size_t)v * kMaxPhases + p];
    std::vector<uint8_t> slot_phase(c->E);
    const std::vector<uint32_t>& ie = *c->hin_edge;
    for (uint32_t i = 0; i < c->E; ++i) slot_phase[i] = edge_phase[ie[i]];
    GMP_TRY(upload(c, c->nph, n_phases, c->N));
    c->max_phases = 0;
    for (uint32_t v = 0; v < c->N; ++v) c->max_phases = std::max<uint32_t>(c->max_phases, n_phases[v]);
    GMP_TRY(upload(c, c->cycle, cycle_ms, c->N));
    GMP_TRY(upload(c, c->offset, offset_ms, c->N));
    GMP_TRY(upload(c, c->green, planes.data(), planes.size()));
    GMP_TRY(upload(c, c->ephase, slot_phase.data(), c->E));
    GMP_CUDA(c, cudaMemsetAsync(c->red, 0, c->N * 4ull * kMaxPhases, c->stream));
    c->red_high = false;
    GMP_TRY(refresh_dynamic(c));
    return sync(c);
}

int gmp_set_red_times(gmp_ctx* c, const uint32_t* red_ms) {
    if (!c || !red_ms) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (!c->own_state) return fail(c, GMP_ERR_STATE, "this context reads another context's traffic state");
    cudaSetDevice(c->device);
    std::vector<uint32_t> planes((size_t)c->N * kMaxPhases);
    bool high = false;  // a non-zero entry in a plane the tick's node pass does not visit
    for (uint32_t v = 0; v < c->N; ++v)
        for (uint32_t p = 0; p < kMaxPhases; ++p) {
            const uint32_t r = red_ms[(size_t)v * kMaxPhases + p];
            planes[(size_t)p * c->N + v] = r;
            high |= p >= c->max_phases && r != 0;
        }
    GMP_TRY(upload(c, c->red, planes.data(), planes.size()));
    c->red_high = high;
    GMP_TRY(refresh_dynamic(c));
    return sync(c);
}

int gmp_set_densities(gmp_ctx* c, const uint32_t* vehicles) {
    if (!c || (!vehicles && c->E)) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (!c->own_state) return fail(c, GMP_ERR_STATE, "this context reads another context's traffic state");
    cudaSetDevice(c->device);
    GMP_TRY(upload(c, c->tick_leave, vehicles, c->E));  // road order, then into slot order
    GMP_CUDA(c, launch_gather_u32(c->stream, c->E, c->in_edge, c->tick_leave, c->veh));
    GMP_TRY(refresh_dynamic(c));
    return sync(c);
}

int gmp_set_densities_async(gmp_ctx* c, const uint32_t* d_vehicles) {
    if (!c || (!d_vehicles && c->E)) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (!c->own_state) return fail(c, GMP_ERR_STATE, "this context reads another context's traffic state");
    cudaSetDevice(c->device);
    GMP_CUDA(c, launch_gather_u32(c->stream, c->E, c->in_edge, d_vehicles, c->veh));
    return refresh_dynamic(c);
}

int gmp_set_params(gmp_ctx* c, const gmp_params* p) {
    if (!c || !p) return GMP_ERR_INVALID_ARG;
    if (p->flags & ~kKnownFlags) return fail(c, GMP_ERR_INVALID_ARG, "unknown flag bits");
    if (p->t_dep_ms >= kTCap) return fail(c, GMP_ERR_INVALID_ARG, "t_dep_ms must be below 2^30");
    if (p->lanes_per_ant && p->lanes_per_ant != 1 && p->lanes_per_ant != 4 && p->lanes_per_ant != 8 &&
        p->lanes_per_ant != 16 && p->lanes_per_ant != 32)
        return fail(c, GMP_ERR_INVALID_ARG, "lanes_per_ant must be 0, 1, 4, 8, 16 or 32");
    if (p->mode > GMP_MODE_PERSISTENT) return fail(c, GMP_ERR_INVALID_ARG, "unknown mode");
    if (p->queue_chunk && p->queue_chunk != 8 && p->queue_chunk != 16 && p->queue_chunk != 32 && p->queue_chunk != 64)
        return fail(c, GMP_ERR_INVALID_ARG, "queue_chunk must be 0, 8, 16, 32 or 64");
    if (p->branches > kMaxBranches) return fail(c, GMP_ERR_INVALID_ARG, "branches must be at most 64");
    if (p->tau_layout > GMP_TAU_SPARSE) return fail(c, GMP_ERR_INVALID_ARG, "unknown tau_layout");
    if (p->max_steps > (1u << 24)) return fail(c, GMP_ERR_INVALID_ARG, "max_steps must be <= 2^24");
    const bool dyn = p->thr_permille != c->prm.thr_permille || p->h_sat_ms != c->prm.h_sat_ms;
    if (dyn && c->has_graph && !c->own_state)
        return fail(c, GMP_ERR_STATE, "the threshold and headway of another context's traffic state are its own");
    c->prm = *p;
    if (dyn && c->has_graph) {
        cudaSetDevice(c->device);
        GMP_TRY(refresh_dynamic(c));
        GMP_TRY(sync(c));
    }
    return GMP_OK;
}

int gmp_get_params(const gmp_ctx* c, gmp_params* p) {
    if (!c || !p) return GMP_ERR_INVALID_ARG;
    *p = c->prm;
    return GMP_OK;
}

}  // extern "C"

namespace {

// Concurrent colony chains of an iterative job with n colonies: params.branches (0 = up to 16).
uint32_t branch_count(const gmp_ctx* c, uint32_t n) {
    if (c->prm.mode == GMP_MODE_PERSISTENT || n == 0) return 1;
    const uint32_t want = c->prm.branches ? c->prm.branches : kDefaultBranches;
    return std::max<uint32_t>(1u, std::min(n, want));
}

// Launch shape of the job for the context's parameters and `total_ants` ants per iteration; `frac` when
// some colony of the job has non-integer exponents.
// The hand-off move count of a job run with kernel configuration kc, or 0 where it does not apply: it
// needs the iterative job, groups that do not step in lockstep, visited sets in shared memory (the tail
// kernel copies them whole), rows of at most eight roads (the pipelined walk's sub-groups) and no road
// from a node to itself (the pipelined walk scores a candidate's row before the candidate is marked
// visited, so such a road would count as a way on; no walk ever takes one).
uint32_t handoff_of(const gmp_ctx* c, const KernelConfig& kc) {
    if (!c->prm.handoff_moves || c->prm.mode == GMP_MODE_PERSISTENT || kc.lockstep || kc.lanes < 4 ||
        !kc.tabu_in_smem || c->maxdeg > 8u || c->self_loops)
        return 0;
    return c->prm.handoff_moves;
}

int job_config(gmp_ctx* c, int lanes, uint64_t total_ants, KernelConfig* kc, bool frac = false) {
    *kc = KernelConfig{};
    const uint32_t ants = (uint32_t)std::min<uint64_t>(total_ants, 0xFFFFFFFFull);
    if (c->prm.mode == GMP_MODE_PERSISTENT) {
        if (lanes == 1) return fail(c, GMP_ERR_UNSUPPORTED, "the persistent job needs 4, 8, 16 or 32 lanes per ant");
        GMP_CUDA(c, persistent_config(c->device, lanes, c->N, c->maxdeg, kc));
    } else if (lanes != 1 && !(c->prm.flags & kFlagNoLockstep) && lockstep_fits(lanes, c->maxdeg)) {
        GMP_CUDA(c, construct_config_lockstep(c->device, lanes, c->N, c->maxdeg, ants, frac, kc));
    } else {
        GMP_CUDA(c, construct_config(c->device, lanes, c->N, c->maxdeg, ants, kc));
    }
    return GMP_OK;
}

// Every device buffer of a job with n colonies, total_ants ants per iteration and at most maxI iterations,
// handed to f(&buffer, entries): reserve_workspace allocates them, workspace_bytes adds them up.
template <class F>
int for_each_workspace(gmp_ctx* c, uint32_t n, uint64_t total_ants, uint32_t maxI, uint64_t log_entries,
                       const KernelConfig& kc, F&& f) {
    Batch& b = c->b;
    const bool persistent = c->prm.mode == GMP_MODE_PERSISTENT;
    const size_t words = (c->N + 31u) / 32u;
    const size_t max_steps = std::max<uint32_t>(default_max_steps(c), 1u);
    GMP_TRY(f(&b.dq, n));
    GMP_TRY(f(&b.prefix, n + 1));
    if (use_sparse(c)) {
        GMP_TRY(f(&b.tflag, (size_t)n * tflag_words(c)));
        GMP_TRY(f(&b.list_e, (size_t)n * c->E));
        GMP_TRY(f(&b.list_tau, (size_t)n * c->E));
    } else {
        GMP_TRY(f(&b.tau, (size_t)n * c->E));
    }
    GMP_TRY(f(&b.th, (size_t)n * c->E));
    GMP_TRY(f(&b.dep, (size_t)n * c->E));
    GMP_TRY(f(&b.qs, n));
    GMP_TRY(f(&b.routes, 2 * (size_t)total_ants * max_steps));  // routes, then their waits
    GMP_TRY(f(&b.ant_steps, (size_t)total_ants));
    GMP_TRY(f(&b.ant_wait, (size_t)total_ants));
    GMP_TRY(f(&b.best_route, (size_t)n * max_steps));
    GMP_TRY(f(&b.route_out, (size_t)n * (max_steps + 1)));
    const uint32_t handoff = handoff_of(c, kc);
    GMP_TRY(f(&b.tickets, (size_t)maxI * branch_count(c, n) * (handoff ? 3u : 1u)));
    if (handoff) {
        GMP_TRY(f(&b.tail_list, (size_t)total_ants));
        GMP_TRY(f(&b.tail_state, (size_t)total_ants));
        GMP_TRY(f(&b.tail_tabu, (size_t)total_ants * words));
    }
    GMP_TRY(f(&b.res, n));
    if (persistent) {
        GMP_TRY(f(&b.ctr, (size_t)n * maxI));
        GMP_TRY(f(&b.qstate, n));
        GMP_TRY(f(&b.qflag, maxI));
    }
    if (persistent || (c->prm.flags & GMP_FLAG_EXACT_H)) GMP_TRY(f(&b.misc, 3));
    if (c->prm.flags & GMP_FLAG_EXACT_H) {
        GMP_TRY(f(&b.hdist, (size_t)n * c->N));
        GMP_TRY(f(&b.hqueue, (size_t)n * 4 * c->N));
        GMP_TRY(f(&b.hstamp, (size_t)n * 2 * c->N));
    }
    if (log_entries) GMP_TRY(f(&b.ant_log, (size_t)log_entries * 4));
    // visited bitmaps in global memory: the job's grid plus one block per concurrent chain (chain grids
    // are shares of the job's grid, rounded up)
    if (!kc.tabu_in_smem) GMP_TRY(f(&b.tabu, ((size_t)kc.grid + branch_count(c, n)) * (kc.block / kc.lanes) * words));
    return GMP_OK;
}

// Device workspace of a job (buffers only grow, so a reservation for the largest job makes later staging
// allocation-free).
int reserve_workspace(gmp_ctx* c, uint32_t n, uint64_t total_ants, uint32_t maxI, uint64_t log_entries,
                      const KernelConfig& kc) {
    Batch& b = c->b;
    if (c->prm.mode == GMP_MODE_PERSISTENT && (uint64_t)kc.grid < n)
        return fail(c, GMP_ERR_UNSUPPORTED, "the persistent job needs at least one resident block per colony");
    // deposit accumulators: zeroed when allocated (or after a job that may have stopped mid-iteration);
    // iterative jobs then keep them zero without clearing them at init
    unsigned long long* dep_before = b.dep;
    const size_t dep_have = dep_before ? c->sizes[(void*)dep_before] : 0;
    GMP_TRY(for_each_workspace(c, n, total_ants, maxI, log_entries, kc,
                               [&](auto** p, size_t count) { return ensure(c, p, count); }));
    if (b.dep != dep_before || c->sizes[(void*)b.dep] != dep_have || b.dep_dirty) {
        GMP_CUDA(c, cudaMemsetAsync(b.dep, 0, c->sizes[(void*)b.dep], c->stream));
        b.dep_dirty = false;
    }
    return GMP_OK;
}

// Bytes the context would hold after reserving the workspace of such a job (nothing is allocated): what it
// holds now, minus each buffer that would be replaced, plus its new size.
uint64_t workspace_bytes(gmp_ctx* c, uint32_t n, uint64_t total_ants, uint32_t maxI, const KernelConfig& kc) {
    uint64_t total = c->used;
    for_each_workspace(c, n, total_ants, maxI, 0, kc, [&](auto** p, size_t count) {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        const auto it = *p ? c->sizes.find((void*)*p) : c->sizes.end();
        const size_t have = it != c->sizes.end() ? it->second : 0;
        if (have < bytes) total += bytes - have;
        return GMP_OK;
    });
    return total;
}

// Split the staged job into concurrent chains of contiguous colonies. Each chain's construction grid is
// its own need, capped at its share (by ants) of the whole job's grid.
int plan_branches(gmp_ctx* c, int lanes, const std::vector<uint32_t>& prefix) {
    Batch& b = c->b;
    b.br.clear();
    b.tabu_used = 0;
    if (b.persistent) {
        if (!b.kc.tabu_in_smem) b.tabu_used = (size_t)b.kc.grid * (b.kc.block / b.kc.lanes) * ((c->N + 31u) / 32u);
        return GMP_OK;
    }
    const uint32_t B = branch_count(c, b.Q);
    const size_t words = (c->N + 31u) / 32u;
    size_t off = 0;
    for (uint32_t j = 0; j < B; ++j) {
        Batch::Branch r{};
        r.q0 = (uint32_t)((uint64_t)b.Q * j / B);
        r.q1 = (uint32_t)((uint64_t)b.Q * (j + 1) / B);
        r.ticket_base = prefix[r.q0];
        r.ants = prefix[r.q1] - prefix[r.q0];
        r.maxI = 0;
        for (uint32_t i = r.q0; i < r.q1; ++i) r.maxI = std::max(r.maxI, b.hq[i].n_iter);
        if (B == 1) {
            r.kc = b.kc;
        } else {
            GMP_TRY(job_config(c, lanes, std::max<uint32_t>(r.ants, 1u), &r.kc, b.kc.frac));
            const uint64_t share = ((uint64_t)b.kc.grid * r.ants + b.total_ants - 1) / std::max<uint32_t>(b.total_ants, 1u);
            r.kc.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)r.kc.grid, share));
        }
        r.tabu_off = off;
        if (!r.kc.tabu_in_smem) off += (size_t)r.kc.grid * (r.kc.block / r.kc.lanes) * words;
        if (b.handoff) GMP_CUDA(c, construct_tail_config(c->device, c->N, std::max<uint32_t>(r.ants, 1u), &r.kc_tail));
        b.br.push_back(r);
    }
    b.tabu_used = off;
    return GMP_OK;
}

}  // namespace

extern "C" {

int gmp_batch_reserve(gmp_ctx* c, uint32_t n, uint64_t total_ants, uint32_t max_iter) {
    if (!c) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (n == 0 || total_ants == 0 || max_iter == 0 || total_ants >= (1ull << 32))
        return fail(c, GMP_ERR_INVALID_ARG, "reserve needs n >= 1, 1 <= total_ants < 2^32, max_iter >= 1");
    cudaSetDevice(c->device);
    GMP_TRY(sync(c));
    KernelConfig kc{};
    GMP_TRY(job_config(c, pick_lanes(c), total_ants, &kc));
    const uint64_t logs = (c->prm.flags & GMP_FLAG_ANT_LOG) ? total_ants * max_iter : 0;
    c->b.staged = c->b.ran = false;  // buffers may move: stage again
    const int rc = reserve_workspace(c, n, total_ants, max_iter, logs, kc);
    if (rc == GMP_ERR_OOM) free_batch(c);  // hold nothing from a reservation that did not fit
    return rc;
}

int gmp_batch_ready(gmp_ctx* c, int* ready) {
    if (!c || !ready) return GMP_ERR_INVALID_ARG;
    if (!c->b.ran || !c->b.done) return fail(c, GMP_ERR_STATE, "launch the batch first");
    const cudaError_t e = cudaEventQuery(c->b.done);
    if (e == cudaErrorNotReady) {
        *ready = 0;
        return GMP_OK;
    }
    GMP_CUDA(c, e);
    *ready = 1;
    return GMP_OK;
}

int gmp_batch_stage(gmp_ctx* c, uint32_t n, const gmp_query* queries) {
    if (!c || (n && !queries)) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (n == 0) return fail(c, GMP_ERR_INVALID_ARG, "empty batch");
    for (uint32_t i = 0; i < n; ++i) GMP_TRY(check_query(c, queries[i], i));
    const int lanes = pick_lanes(c);
    if ((uint32_t)construct_max_degree(lanes) < c->maxdeg || c->maxdeg > 128u)
        return fail(c, GMP_ERR_UNSUPPORTED, "out-degree %u exceeds %d for %d lanes per ant", c->maxdeg,
                    construct_max_degree(lanes), lanes);
    if (lanes == 1 && !construct_thread_fits(c->N))
        return fail(c, GMP_ERR_UNSUPPORTED, "one thread per ant needs the visited bitmaps in shared memory "
                                            "(N <= 25600)");
    cudaSetDevice(c->device);
    GMP_TRY(sync(c));
    Batch& b = c->b;
    b.hq.assign(queries, queries + n);
    b.Q = n;
    b.max_steps = std::max<uint32_t>(default_max_steps(c), 1u);
    std::vector<DevQuery> hdq(n);
    std::vector<uint32_t> prefix(n + 1, 0);
    uint64_t total = 0, logs = 0;
    uint32_t maxI = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const gmp_query& q = queries[i];
        DevQuery& d = hdq[i];
        memset(&d, 0, sizeof d);
        d.src = q.src;
        d.dst = q.dst;
        d.n_ants = q.n_ants;
        d.n_iter = q.n_iter;
        d.ant_base = (uint32_t)total;
        d.active = q.src != q.dst;
        set_exponents(d, q.alpha, q.beta);
        d.rho_fix = (uint64_t)nearbyint(ldexp((double)q.rho, 32));
        d.seed = q.seed;
        d.log_base = logs;
        prefix[i] = (uint32_t)total;
        total += q.n_ants;
        logs += (uint64_t)q.n_ants * q.n_iter;
        maxI = std::max(maxI, q.n_iter);
        if (total >= (1ull << 32)) return fail(c, GMP_ERR_INVALID_ARG, "batch holds 2^32 or more ants");
    }
    prefix[n] = (uint32_t)total;
    for (uint32_t i = 0; i < n; ++i) {  // destination coordinates for the heuristic
        hdq[i].xd = c->hx[queries[i].dst];
        hdq[i].yd = c->hy[queries[i].dst];
    }
    b.total_ants = (uint32_t)total;
    b.maxI = maxI;
    b.log_entries = (c->prm.flags & GMP_FLAG_ANT_LOG) ? logs : 0;
    b.persistent = c->prm.mode == GMP_MODE_PERSISTENT;
    b.exact_h = (c->prm.flags & GMP_FLAG_EXACT_H) != 0;
    b.queue_general = c->max_phases > 2;
    if (c->prm.tau_layout == GMP_TAU_SPARSE && (b.persistent || (c->prm.flags & GMP_FLAG_RANDOM_TAU)))
        return fail(c, GMP_ERR_UNSUPPORTED, "the sparse pheromone layout needs the iterative job and 1.0 initial pheromone");
    b.sparse = use_sparse(c);
    bool frac = false;
    for (uint32_t i = 0; i < n; ++i) frac = frac || (hdq[i].active & kQueryFracExp) != 0u;
    GMP_TRY(job_config(c, lanes, b.total_ants, &b.kc, frac));
    b.handoff = handoff_of(c, b.kc);
    GMP_TRY(plan_branches(c, lanes, prefix));
    GMP_TRY(reserve_workspace(c, n, b.total_ants, maxI, b.log_entries, b.kc));
    GMP_TRY(upload(c, b.dq, hdq.data(), n));
    GMP_TRY(upload(c, b.prefix, prefix.data(), n + 1));
    GMP_TRY(sync(c));
    b.staged = true;
    b.ran = false;
    return GMP_OK;
}

namespace {

// Per-kernel timing events for the staged job (created when the timing flag is set).
int prepare_events(gmp_ctx* c) {
    Batch& b = c->b;
    const bool timed = (c->prm.flags & kFlagKernelTiming) != 0;
    const size_t n_ev = timed ? job_event_count(b) : 0;
    if (b.ev.size() != n_ev || b.timed != timed) {
        drop_graph(b);
        drop_events(b);
        b.ev.resize(n_ev);
        for (size_t i = 0; i < n_ev; ++i) GMP_CUDA(c, cudaEventCreate(&b.ev[i]));
        b.timed = timed;
    }
    return GMP_OK;
}

// The staged job was launched (by itself or inside a multi-graph launch): mark its completion point
// on the context's stream.
int mark_launched(gmp_ctx* c) {
    Batch& b = c->b;
    if (!b.done) GMP_CUDA(c, cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
    GMP_CUDA(c, cudaEventRecord(b.done, c->stream));
    b.ran = true;
    return GMP_OK;
}

}  // namespace

int gmp_batch_launch(gmp_ctx* c) {
    if (!c) return GMP_ERR_INVALID_ARG;
    Batch& b = c->b;
    if (!b.staged) return fail(c, GMP_ERR_STATE, "stage a batch first");
    cudaSetDevice(c->device);
    GMP_TRY(prepare_events(c));
    if (c->prm.flags & kFlagNoGraph) {
        GMP_TRY(enqueue_job(c));
    } else {
        const BatchKey k = key_of(c);
        if (!b.exec || !(b.key == k) || !same_plan(b.br, b.exec_br)) {
            // capture the job; an executable graph of the same topology (chain count, iterations per
            // chain, kernel shapes) is updated in place with the new parameters, which costs far less
            // than instantiating one (jobs of a server change shape with every batch)
            cudaGraph_t g = nullptr;
            GMP_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue_job(c);
            const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
            if (rc != GMP_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            GMP_CUDA(c, ce);
            const std::vector<uint32_t> sig = topology_of(b);
            b.exec = nullptr;
            auto hit = b.execs.find(sig);
            if (hit != b.execs.end()) {
                cudaGraphExecUpdateResultInfo info{};
                if (cudaGraphExecUpdate(hit->second, g, &info) == cudaSuccess) {
                    b.exec = hit->second;
                } else {
                    cudaGetLastError();
                    cudaGraphExecDestroy(hit->second);
                    b.execs.erase(hit);
                }
            }
            if (!b.exec) {
                if (b.execs.size() >= kMaxCachedGraphs) drop_graph(b);
                const cudaError_t ie = cudaGraphInstantiate(&b.exec, g, 0);
                if (ie != cudaSuccess) {
                    b.exec = nullptr;
                    cudaGraphDestroy(g);
                    GMP_CUDA(c, ie);
                }
                b.execs[sig] = b.exec;
            }
            cudaGraphDestroy(g);
            b.key = k;
            b.exec_br = b.br;
        }
        GMP_CUDA(c, cudaGraphLaunch(b.exec, c->stream));
    }
    return mark_launched(c);
}

int gmp_batch_collect(gmp_ctx* c, gmp_result* results) {
    if (!c || !results) return GMP_ERR_INVALID_ARG;
    Batch& b = c->b;
    if (!b.ran) return fail(c, GMP_ERR_STATE, "launch the batch first");
    cudaSetDevice(c->device);
    std::vector<DevResult> hr(b.Q);
    GMP_CUDA(c, cudaMemcpyAsync(hr.data(), b.res, b.Q * sizeof(DevResult), cudaMemcpyDeviceToHost, c->stream));
    uint32_t misc[3] = {0, 0, 0};
    if (b.persistent || b.exact_h)
        GMP_CUDA(c, cudaMemcpyAsync(misc, b.misc, sizeof misc, cudaMemcpyDeviceToHost, c->stream));
    GMP_TRY(sync(c));
    if (b.persistent && misc[1]) {
        b.dep_dirty = true;
        return fail(c, GMP_ERR_TIMEOUT, "a bounded device wait of the persistent job expired");
    }
    if (b.exact_h && misc[2]) return fail(c, GMP_ERR_TIMEOUT, "the exact heuristic's relaxation passed its level bound");
    for (uint32_t i = 0; i < b.Q; ++i) {
        gmp_result& r = results[i];
        const DevResult& d = hr[i];
        r.route_len = d.route_len;
        r.travel_ms = d.travel_ms;
        r.wait_ms = d.wait_ms;
        r.ant_steps = d.ant_steps;
        r.n_success = d.n_success;
        r.best_iter = d.best_iter;
        r.best_ant = d.best_ant;
        r.status = d.status;
        if (d.status == GMP_OK) {
            if (!r.route || r.route_cap < d.route_len) {
                r.status = GMP_ERR_BUFFER;
            } else {
                GMP_CUDA(c, cudaMemcpyAsync(r.route, b.route_out + (size_t)i * (b.max_steps + 1),
                                            d.route_len * 4ull, cudaMemcpyDeviceToHost, c->stream));
            }
        }
    }
    return sync(c);
}

int gmp_solve_batch(gmp_ctx* c, uint32_t n, const gmp_query* queries, gmp_result* results) {
    GMP_TRY(gmp_batch_stage(c, n, queries));
    GMP_TRY(gmp_batch_launch(c));
    return gmp_batch_collect(c, results);
}

int gmp_solve(gmp_ctx* c, uint32_t src, uint32_t dst, uint32_t n_ants, uint32_t n_iter, float alpha, float beta,
              float rho, uint64_t seed, gmp_result* out) {
    if (!out) return GMP_ERR_INVALID_ARG;
    gmp_query q;
    memset(&q, 0, sizeof q);
    q.src = src;
    q.dst = dst;
    q.n_ants = n_ants;
    q.n_iter = n_iter;
    q.alpha = alpha;
    q.beta = beta;
    q.rho = rho;
    q.seed = seed;
    const int rc = gmp_solve_batch(c, 1, &q, out);
    if (rc != GMP_OK) {
        out->status = rc;
        return rc;
    }
    return out->status;
}

int gmp_get_pheromone(gmp_ctx* c, uint32_t slot, uint64_t* out_tau) {
    if (!c || !out_tau) return GMP_ERR_INVALID_ARG;
    if (!c->b.ran) return fail(c, GMP_ERR_STATE, "no batch has run");
    if (slot >= c->b.Q) return fail(c, GMP_ERR_INVALID_ARG, "slot out of range");
    cudaSetDevice(c->device);
    Batch& b = c->b;
    if (!b.sparse) {
        GMP_CUDA(c, cudaMemcpyAsync(out_tau, b.tau + (size_t)slot * c->E, c->E * 8ull, cudaMemcpyDeviceToHost,
                                    c->stream));
        return sync(c);
    }
    // sparse layout: the baseline on every road, then the registered roads' own values
    uint64_t* tmp = nullptr;
    GMP_TRY(dalloc(c, &tmp, c->E));
    const size_t co = (size_t)slot * c->E;
    int rc = GMP_OK;
    if (launch_materialize_tau(c->stream, c->E, b.qs + slot, b.list_e + co, b.list_tau + co, tmp) != cudaSuccess ||
        cudaMemcpyAsync(out_tau, tmp, c->E * 8ull, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rc = fail(c, GMP_ERR_CUDA, "reading the sparse pheromone table failed");
    if (rc == GMP_OK) rc = sync(c);
    sync(c);
    dfree(c, &tmp);
    return rc;
}

int gmp_get_ant_log(gmp_ctx* c, uint32_t slot, uint32_t* out, uint64_t capacity_entries) {
    if (!c || !out) return GMP_ERR_INVALID_ARG;
    Batch& b = c->b;
    if (!b.ran || !b.log_entries) return fail(c, GMP_ERR_STATE, "no ant log (set GMP_FLAG_ANT_LOG before staging)");
    if (slot >= b.Q) return fail(c, GMP_ERR_INVALID_ARG, "slot out of range");
    const gmp_query& q = b.hq[slot];
    const uint64_t n = (uint64_t)q.n_ants * q.n_iter * 4;
    if (capacity_entries < n) return fail(c, GMP_ERR_BUFFER, "need %llu entries", (unsigned long long)n);
    uint64_t base = 0;
    for (uint32_t i = 0; i < slot; ++i) base += (uint64_t)b.hq[i].n_ants * b.hq[i].n_iter;
    cudaSetDevice(c->device);
    GMP_CUDA(c, cudaMemcpyAsync(out, b.ant_log + base * 4, n * 4, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

int gmp_get_phase_order(gmp_ctx* c, uint8_t* out) {
    if (!c || !out) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    cudaSetDevice(c->device);
    GMP_CUDA(c, cudaMemcpyAsync(out, c->order, (size_t)c->N * kMaxPhases, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

int gmp_get_densities(gmp_ctx* c, uint32_t* vehicles) {
    if (!c || (!vehicles && c->E)) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    cudaSetDevice(c->device);
    std::vector<uint32_t> slots(c->E);
    if (c->E) GMP_CUDA(c, cudaMemcpyAsync(slots.data(), c->veh, c->E * 4ull, cudaMemcpyDeviceToHost, c->stream));
    GMP_TRY(sync(c));
    const std::vector<uint32_t>& ie = *c->hin_edge;
    for (uint32_t i = 0; i < c->E; ++i) vehicles[ie[i]] = slots[i];
    return GMP_OK;
}

int gmp_get_red_times(gmp_ctx* c, uint32_t* red_ms) {
    if (!c || !red_ms) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    cudaSetDevice(c->device);
    std::vector<uint32_t> planes((size_t)c->N * kMaxPhases);
    GMP_CUDA(c, cudaMemcpyAsync(planes.data(), c->red, planes.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    GMP_TRY(sync(c));
    for (uint32_t v = 0; v < c->N; ++v)
        for (uint32_t p = 0; p < kMaxPhases; ++p) red_ms[(size_t)v * kMaxPhases + p] = planes[(size_t)p * c->N + v];
    return GMP_OK;
}

int gmp_tick(gmp_ctx* c, uint64_t t_now_ms, uint32_t dt_ms) {
    if (!c) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    if (!c->own_state) return fail(c, GMP_ERR_STATE, "this context reads another context's traffic state");
    if (t_now_ms > kTickClockMax || dt_ms > kTickDtMax)
        return fail(c, GMP_ERR_INVALID_ARG, "tick clock must be <= 2^48 ms and dt <= 2^30 ms");
    cudaSetDevice(c->device);
    const QueueTables t = queue_tables(c);
    GMP_CUDA(c, launch_tick_node(c->stream, t, t_now_ms, dt_ms, c->max_phases, c->tick_leave, c->tick_K));
    if (c->red_high) {  // the planes the node pass does not visit: every phase there is >= the node's count
        GMP_CUDA(c, cudaMemsetAsync(c->red + (size_t)c->max_phases * c->N, 0,
                                    (size_t)(kMaxPhases - c->max_phases) * c->N * 4, c->stream));
        c->red_high = false;
    }
    GMP_CUDA(c, launch_queue(c->stream, t, c->max_phases, QueuePass::kTick));
    return GMP_OK;
}

int gmp_get_edge_times(gmp_ctx* c, uint32_t* tt_ms, uint32_t* qd_ms) {
    if (!c) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    std::vector<EdgeRec> h(c->E);
    cudaSetDevice(c->device);
    if (c->E) GMP_CUDA(c, cudaMemcpyAsync(h.data(), c->rec, c->E * sizeof(EdgeRec), cudaMemcpyDeviceToHost, c->stream));
    GMP_TRY(sync(c));
    for (uint32_t e = 0; e < c->E; ++e) {
        if (tt_ms) tt_ms[e] = h[e].tt;
        if (qd_ms) qd_ms[e] = h[e].qd_fl & kQdMask;
    }
    return GMP_OK;
}

int gmp_get_kernel_times(gmp_ctx* c, float* out) {
    if (!c || !out) return GMP_ERR_INVALID_ARG;
    Batch& b = c->b;
    for (int i = 0; i < 5; ++i) out[i] = 0.0f;
    if (!b.ran || !b.timed || b.ev.empty()) return fail(c, GMP_ERR_STATE, "no timed job has run");
    cudaSetDevice(c->device);
    GMP_TRY(sync(c));
    float ms = 0;
    if (b.persistent) {  // construction, evaporation, best tracking and queue update run in one kernel
        GMP_CUDA(c, cudaEventElapsedTime(&ms, b.ev[1], b.ev[2]));
        out[0] = ms;
        GMP_CUDA(c, cudaEventElapsedTime(&ms, b.ev[0], b.ev[3]));
        out[4] = ms;
        return GMP_OK;
    }
    for (size_t j = 0; j < b.br.size(); ++j) {  // summed over chains (concurrent chains overlap)
        const size_t eb = branch_event_base(b, j);
        for (uint32_t it = 0; it < b.br[j].maxI; ++it) {
            const size_t prev = eb + 2 * (size_t)it;
            for (int k = 0; k < 2; ++k) {
                GMP_CUDA(c, cudaEventElapsedTime(&ms, b.ev[prev + k], b.ev[prev + k + 1]));
                out[k] += ms;
            }
        }
    }
    GMP_CUDA(c, cudaEventElapsedTime(&ms, b.ev[0], b.ev[1]));
    out[2] = ms;
    GMP_CUDA(c, cudaEventElapsedTime(&ms, b.ev[2], b.ev[3]));
    out[2] += ms;
    GMP_CUDA(c, cudaEventElapsedTime(&ms, b.ev[0], b.ev[3]));
    out[4] = ms;
    return GMP_OK;
}

int gmp_get_launch_count(const gmp_ctx* c, uint64_t* out) {
    if (!c || !out) return GMP_ERR_INVALID_ARG;
    *out = c->b.launches;
    return GMP_OK;
}

}  // extern "C"

// =====================================================================================================
// gmp_multi: the staged jobs of several contexts (one road graph each) as one captured launch.
// =====================================================================================================
struct gmp_multi {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> joins, pre;
    cudaGraphExec_t exec = nullptr;
    struct Member {
        gmp_ctx* c;
        cudaStream_t st;
        BatchKey key;
        std::vector<Batch::Branch> plan;
    };
    std::vector<Member> members;  // what `exec` was captured from
    std::string err;
};

namespace {

int mfail(gmp_multi* m, int code, const std::string& msg) {
    m->err = msg;
    return code;
}

bool same_members(const gmp_multi* m, gmp_ctx* const* ctxs, uint32_t n) {
    if (m->members.size() != n) return false;
    for (uint32_t i = 0; i < n; ++i) {
        const gmp_multi::Member& x = m->members[i];
        if (x.c != ctxs[i] || x.st != ctxs[i]->stream || !(x.key == key_of(ctxs[i])) ||
            !same_plan(x.plan, ctxs[i]->b.br))
            return false;
    }
    return true;
}

}  // namespace

extern "C" {

int gmp_multi_create(gmp_multi** out, int device) {
    if (!out) return GMP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GMP_ERR_CUDA;
    }
    gmp_multi* m = new gmp_multi();
    m->device = device;
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        gmp_multi_destroy(m);
        return GMP_ERR_CUDA;
    }
    *out = m;
    return GMP_OK;
}

void gmp_multi_destroy(gmp_multi* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->exec) cudaGraphExecDestroy(m->exec);
    for (cudaEvent_t e : m->joins) cudaEventDestroy(e);
    for (cudaEvent_t e : m->pre) cudaEventDestroy(e);
    if (m->fork) cudaEventDestroy(m->fork);
    if (m->done) cudaEventDestroy(m->done);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

const char* gmp_multi_last_error(const gmp_multi* m) { return m ? m->err.c_str() : "null handle"; }

int gmp_multi_launch(gmp_multi* m, gmp_ctx* const* ctxs, uint32_t n) {
    if (!m || !ctxs || n == 0) return GMP_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    for (uint32_t i = 0; i < n; ++i) {
        gmp_ctx* c = ctxs[i];
        if (!c) return mfail(m, GMP_ERR_INVALID_ARG, "null context");
        if (c->device != m->device) return mfail(m, GMP_ERR_INVALID_ARG, "contexts must be on the handle's device");
        if (!c->b.staged) return mfail(m, GMP_ERR_STATE, "every context needs a staged batch");
        if (c->b.persistent) return mfail(m, GMP_ERR_UNSUPPORTED, "the multi-graph launch runs iterative jobs");
        for (uint32_t j = 0; j < i; ++j)
            if (ctxs[j] == c) return mfail(m, GMP_ERR_INVALID_ARG, "a context appears twice");
        const int rc = prepare_events(c);
        if (rc != GMP_OK) return mfail(m, rc, c->err);
        const int rb = ensure_branch_streams(c, c->b.br.size() > 1 ? c->b.br.size() : 0);
        if (rb != GMP_OK) return mfail(m, rb, c->err);
    }
    while (m->joins.size() < n) {
        cudaEvent_t e = nullptr, p = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (e) cudaEventDestroy(e);
            return mfail(m, GMP_ERR_CUDA, "cudaEventCreate failed");
        }
        m->joins.push_back(e);
        m->pre.push_back(p);
    }
    if (!m->exec || !same_members(m, ctxs, n)) {
        if (m->exec) {
            cudaGraphExecDestroy(m->exec);
            m->exec = nullptr;
        }
        m->members.clear();
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return mfail(m, GMP_ERR_CUDA, cudaGetErrorString(ce));
        int rc = cudaEventRecord(m->fork, m->stream) == cudaSuccess ? GMP_OK : GMP_ERR_CUDA;
        for (uint32_t i = 0; i < n && rc == GMP_OK; ++i) {
            gmp_ctx* c = ctxs[i];
            if (cudaStreamWaitEvent(c->stream, m->fork, 0) != cudaSuccess) {
                rc = GMP_ERR_CUDA;
                break;
            }
            rc = enqueue_job(c);
            if (rc != GMP_OK) {
                m->err = c->err;
                break;
            }
            if (cudaEventRecord(m->joins[i], c->stream) != cudaSuccess ||
                cudaStreamWaitEvent(m->stream, m->joins[i], 0) != cudaSuccess)
                rc = GMP_ERR_CUDA;
        }
        ce = cudaStreamEndCapture(m->stream, &g);
        if (rc != GMP_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return mfail(m, rc != GMP_OK ? rc : GMP_ERR_CUDA, rc != GMP_OK ? m->err : cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&m->exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            m->exec = nullptr;
            return mfail(m, GMP_ERR_CUDA, cudaGetErrorString(ce));
        }
        for (uint32_t i = 0; i < n; ++i)
            m->members.push_back(gmp_multi::Member{ctxs[i], ctxs[i]->stream, key_of(ctxs[i]), ctxs[i]->b.br});
    }
    // the launch waits for work already queued on every context's stream; each context's stream then
    // waits for the launch, so gmp_batch_ready / gmp_batch_collect work per context as usual
    for (uint32_t i = 0; i < n; ++i) {
        if (cudaEventRecord(m->pre[i], ctxs[i]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(m->stream, m->pre[i], 0) != cudaSuccess)
            return mfail(m, GMP_ERR_CUDA, "ordering after the contexts' streams failed");
    }
    cudaError_t le = cudaGraphLaunch(m->exec, m->stream);
    if (le != cudaSuccess) return mfail(m, GMP_ERR_CUDA, cudaGetErrorString(le));
    if (cudaEventRecord(m->done, m->stream) != cudaSuccess) return mfail(m, GMP_ERR_CUDA, "event record failed");
    for (uint32_t i = 0; i < n; ++i) {
        gmp_ctx* c = ctxs[i];
        if (cudaStreamWaitEvent(c->stream, m->done, 0) != cudaSuccess)
            return mfail(m, GMP_ERR_CUDA, "ordering the contexts after the launch failed");
        const int rc = mark_launched(c);
        if (rc != GMP_OK) return mfail(m, rc, c->err);
    }
    return GMP_OK;
}

}  // extern "C"

// =====================================================================================================
// gmp_solve_static: one colony without any device allocation by the call.
//
// Some callers cannot allocate device memory when they solve: code running where cudaMalloc is
// forbidden or unsafe (inside a latency-critical loop that must never block on the allocator, under a
// device memory pool or quota that is already spent, or from a framework that owns all allocations).
// For them this entry point keeps every temporary of the colony in one file-scope device array of
// GMP_STATIC_SCRATCH_BYTES and writes the result into buffers the caller already owns. The array
// exists on every GPU that loads the library, for the life of the process. Its device address is
// looked up once per device, by the first call on that device, which should therefore come before
// any stream capture. All calls share the array and it keeps the last call's contents: every call
// re-initialises what must start from zero or from its initial value, and calls whose work overlaps
// on the GPU (for example on two streams) race on it.
// =====================================================================================================
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[GMP_STATIC_SCRATCH_BYTES];

constexpr int kStaticMaxDevices = 64;
// Device address of the array on each device, looked up once per device (call_once keeps two host
// threads making their first call on a device at the same time from racing on the entry).
void* g_static_ptr[kStaticMaxDevices] = {nullptr};
std::once_flag g_static_once[kStaticMaxDevices];
cudaError_t g_static_err[kStaticMaxDevices] = {};

__global__ void k_static_query(DevQuery q, DevQuery* __restrict__ dq, uint32_t* __restrict__ prefix) {
    dq[0] = q;
    prefix[0] = 0;
    prefix[1] = q.n_ants;
}

size_t align256(size_t n) { return (n + 255u) & ~(size_t)255u; }

}  // namespace

extern "C" int gmp_solve_static(gmp_ctx* c, uint32_t src, uint32_t dst, uint32_t n_ants, uint32_t n_iter, float alpha,
                                float beta, float rho, uint64_t seed, gmp_device_result* d_result, uint32_t* d_route,
                                uint32_t route_cap) {
    static_assert(sizeof(gmp_device_result) == sizeof(DevResult), "result row layout");
    if (!c || !d_result || !d_route) return GMP_ERR_INVALID_ARG;
    if (!c->has_graph) return fail(c, GMP_ERR_STATE, "load a graph first");
    gmp_query qq;
    memset(&qq, 0, sizeof qq);
    qq.src = src;
    qq.dst = dst;
    qq.n_ants = n_ants;
    qq.n_iter = n_iter;
    qq.alpha = alpha;
    qq.beta = beta;
    qq.rho = rho;
    qq.seed = seed;
    GMP_TRY(check_query(c, qq, 0));
    if (c->prm.flags & GMP_FLAG_EXACT_H)
        return fail(c, GMP_ERR_UNSUPPORTED, "the allocation-free solve has no room for the exact heuristic");
    if (c->device < 0 || c->device >= kStaticMaxDevices) return fail(c, GMP_ERR_UNSUPPORTED, "device index too high");
    const int lanes = pick_lanes(c);
    if ((uint32_t)construct_max_degree(lanes) < c->maxdeg || c->maxdeg > 128u || lanes == 1)
        return fail(c, GMP_ERR_UNSUPPORTED, "out-degree %u is beyond the static solve's kernels", c->maxdeg);
    GMP_CUDA(c, cudaSetDevice(c->device));
    std::call_once(g_static_once[c->device], [&] {  // first call on this device: where the array lives
        void* p = nullptr;
        g_static_err[c->device] = cudaGetSymbolAddress(&p, g_static_scratch);
        g_static_ptr[c->device] = p;
    });
    GMP_CUDA(c, g_static_err[c->device]);
    const uint32_t S = std::max<uint32_t>(default_max_steps(c), 1u);
    const uint32_t route_need = std::min<uint32_t>(c->N, S + 1u);  // nodes of the longest possible route
    if (route_cap < route_need)
        return fail(c, GMP_ERR_BUFFER, "route buffer needs %u entries (min(N, max_steps + 1))", route_need);
    KernelConfig kc{};
    if (!(c->prm.flags & kFlagNoLockstep) && lockstep_fits(lanes, c->maxdeg))
        GMP_CUDA(c, construct_config_lockstep(c->device, lanes, c->N, c->maxdeg, n_ants,
                                              floorf(alpha) != alpha || floorf(beta) != beta, &kc));
    else
        GMP_CUDA(c, construct_config(c->device, lanes, c->N, c->maxdeg, n_ants, &kc));
    // carve the scratch array
    const size_t E = c->E, words = (c->N + 31u) / 32u;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t o_dq = take(sizeof(DevQuery)), o_prefix = take(8), o_qs = take(sizeof(QueryState));
    const size_t o_tickets = take((size_t)n_iter * 4), o_tau = take(E * 8), o_th = take(E * 8), o_dep = take(E * 8);
    const size_t o_routes = take((size_t)n_ants * S * 8), o_steps = take((size_t)n_ants * 4);  // routes, waits
    const size_t o_wait = take((size_t)n_ants * 4), o_best = take((size_t)S * 4);
    const size_t o_tabu = kc.tabu_in_smem ? 0 : take((size_t)kc.grid * (kc.block / kc.lanes) * words * 4);
    if (off > GMP_STATIC_SCRATCH_BYTES)
        return fail(c, GMP_ERR_BUFFER, "this colony needs %zu bytes of static scratch, the limit is %llu", off,
                    (unsigned long long)GMP_STATIC_SCRATCH_BYTES);
    unsigned char* base = static_cast<unsigned char*>(g_static_ptr[c->device]);
    DevQuery* dq = reinterpret_cast<DevQuery*>(base + o_dq);
    uint32_t* prefix = reinterpret_cast<uint32_t*>(base + o_prefix);
    QueryState* qs = reinterpret_cast<QueryState*>(base + o_qs);
    uint32_t* tickets = reinterpret_cast<uint32_t*>(base + o_tickets);
    uint64_t* tau = reinterpret_cast<uint64_t*>(base + o_tau);
    uint2* th = reinterpret_cast<uint2*>(base + o_th);
    unsigned long long* dep = reinterpret_cast<unsigned long long*>(base + o_dep);
    uint32_t* routes = reinterpret_cast<uint32_t*>(base + o_routes);
    uint32_t* ant_steps = reinterpret_cast<uint32_t*>(base + o_steps);
    uint32_t* ant_wait = reinterpret_cast<uint32_t*>(base + o_wait);
    uint32_t* best_route = reinterpret_cast<uint32_t*>(base + o_best);
    uint32_t* tabu = kc.tabu_in_smem ? nullptr : reinterpret_cast<uint32_t*>(base + o_tabu);
    DevQuery hq{};
    hq.src = src;
    hq.dst = dst;
    hq.n_ants = n_ants;
    hq.n_iter = n_iter;
    hq.ant_base = 0;
    hq.active = src != dst;
    set_exponents(hq, alpha, beta);
    hq.rho_fix = (uint64_t)nearbyint(ldexp((double)rho, 32));
    hq.seed = seed;
    hq.xd = c->hx[dst];
    hq.yd = c->hy[dst];
    hq.log_base = 0;
    cudaStream_t s = c->stream;
    k_static_query<<<1, 1, 0, s>>>(hq, dq, prefix);
    GMP_CUDA(c, cudaGetLastError());
    // init clears the pheromone, deposits, colony state and ticket counters left by the previous call
    GMP_CUDA(c, launch_init_batch(s, 1, c->E, dq, c->col, c->x, c->y, c->kappa, c->prm.flags, tau, th, dep,
                                  qs, tickets, n_iter, 0u, nullptr, 0u, nullptr, c->N, true));
    if (tabu)  // global visited bitmaps start clean; each walk clears its own bits when it ends
        GMP_CUDA(c, cudaMemsetAsync(tabu, 0, (size_t)kc.grid * (kc.block / kc.lanes) * words * 4, s));
    ConstructArgs a{};
    a.rec = c->rec;
    a.row_ptr = c->row_ptr;
    a.col = c->col;
    a.queries = dq;
    a.ant_prefix = prefix;
    a.tau = tau;
    a.th = th;
    a.dep = dep;
    a.qs = qs;
    a.routes = routes;
    a.rwait = routes + (size_t)n_ants * S;
    a.ant_steps = ant_steps;
    a.ant_wait = ant_wait;
    a.ant_log = nullptr;
    a.tickets = tickets;
    a.tabu_global = tabu;
    a.n_queries = 1;
    a.total_ants = n_ants;
    a.n_edges = c->E;
    a.max_steps = S;
    a.tabu_words = (uint32_t)words;
    a.t_dep = c->prm.t_dep_ms;
    a.thr_on = c->prm.thr_permille != kThrOff;
    a.tabu_in_smem = kc.tabu_in_smem ? 1u : 0u;
    a.kappa = c->kappa;
    IterEndArgs e = iter_end_args(c, 1, dq, tau, th, dep, qs, routes, ant_steps, ant_wait, best_route, S);
    for (uint32_t it = 0; it < n_iter; ++it) {
        GMP_CUDA(c, launch_construct(s, kc, a, it));
        e.it = it;
        GMP_CUDA(c, launch_iter_end(s, e));
        if (c->max_phases > 2)  // the iteration end updated the intersections with <= 2 phases only
            GMP_CUDA(c, launch_queue_general(s, e.qt, QueuePass::kIterate));
    }
    GMP_CUDA(c, launch_finalize(s, 1, dq, qs, best_route, c->col, S, reinterpret_cast<DevResult*>(d_result), d_route));
    return GMP_OK;
}

namespace gmp {

int ctx_check_query(gmp_ctx* c, const gmp_query& q) { return check_query(c, q, 0); }

void ctx_set_stream_alloc(gmp_ctx* c) { c->stream_alloc = true; }

int ctx_rebind_state(gmp_ctx* c, gmp_ctx* holder) {
    if (c->own_state || !c->lender || !holder->own_state)
        return fail(c, GMP_ERR_STATE, "only a view of another context's traffic state can be moved to another");
    if ((holder->lender ? holder->lender : holder) != c->lender)
        return fail(c, GMP_ERR_INVALID_ARG, "the traffic state belongs to another road graph");
    if (c->state_lender == holder) return GMP_OK;
    --c->state_lender->views;
    ++holder->views;
    c->state_lender = holder;
    c->order = holder->order;
    c->red = holder->red;
    c->veh = holder->veh;
    c->rec = holder->rec;
    c->tick_leave = holder->tick_leave;
    c->tick_K = holder->tick_K;
    return GMP_OK;
}

cudaEvent_t ctx_done_event(const gmp_ctx* c) { return c->b.ran ? c->b.done : nullptr; }

bool ctx_owns_state(const gmp_ctx* c) { return c->own_state; }

int ctx_copy_state(gmp_ctx* dst, const gmp_ctx* src) {
    cudaSetDevice(dst->device);
    return copy_state(dst, src);
}

uint64_t ctx_job_bytes(gmp_ctx* c, uint32_t n, uint64_t total_ants, uint32_t max_iter) {
    KernelConfig kc{};
    if (job_config(c, pick_lanes(c), total_ants, &kc) != GMP_OK) return ~0ull;
    return workspace_bytes(c, n, total_ants, max_iter, kc);
}

}  // namespace gmp

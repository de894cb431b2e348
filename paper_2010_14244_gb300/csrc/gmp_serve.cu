// Route server with continuous batching (gmp_server_*, declared in include/gmacop.h).
//
// The paper routes vehicles one request at a time (Fig. 3); a deployment receives route requests
// continuously while the traffic state changes. The server keeps one road graph and its traffic state
// resident on the device and runs colonies as they arrive:
//   - one road graph: the caller's context holds it; every slot is a view of it (gmp_share_graph), so
//     the static arrays exist once on the GPU whatever the number of slots;
//   - two versions of the traffic state: the caller's and a copy the server keeps. A tick copies the
//     current version into the other one and advances that copy in place, on its own stream, after
//     the jobs still reading the version it overwrites; jobs launched afterwards run on the new version
//     (their streams wait for the tick). Running jobs never wait for a tick, nor a tick for them beyond
//     the previous version's jobs;
//   - slots: each slot has its own batch workspace and CUDA stream, so jobs of different slots overlap
//     on the GPU; workspaces grow through the stream-ordered allocator (no device-wide synchronisation);
//   - admission by memory, per job: when a slot is idle it takes what waits at the head of the queue,
//     up to max_batch requests, cut down until the job's workspace fits both the server's memory budget
//     (shared by all slots) and the memory the GPU has free at that moment; requests that do not fit
//     wait for a later job;
//   - continuous batching: every pump collects finished jobs and starts jobs on idle slots at once.
// A request's result depends only on the request and the traffic state it ran on (Philox streams are
// keyed by the request's own seed), so it is the same alone and in any mix. The server is
// single-threaded: the caller drives it with gmp_server_pump.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <string>
#include <vector>

#include "gmacop.h"
#include "gmp_internal.h"

using namespace gmp;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    gmp_query q;
    uint64_t tag, t_submit;
};

struct Slot {
    gmp_ctx* ctx = nullptr;  // a view of the road graph with a batch workspace of its own
    bool busy = false;
    uint32_t version = 0;  // traffic-state version its job runs on
    std::vector<Request> job;
    uint64_t t_launch = 0, clock_ms = 0;
    std::vector<uint32_t> routes;  // job.size() * route_cap
    std::vector<gmp_result> res;
};

struct Done {
    gmp_served s;
    std::vector<uint32_t> route;
};

}  // namespace

struct gmp_server {
    gmp_ctx* state[2] = {nullptr, nullptr};     // [0] the caller's context, [1] the server's copy
    cudaEvent_t ready[2] = {nullptr, nullptr};  // recorded after the tick that produced each version
    bool has_ready[2] = {false, false};
    uint32_t cur = 0;  // the version new jobs run on
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::deque<Done> done;
    gmp_server_config cfg{};
    uint64_t budget = 0;     // bytes all slots' workspaces may hold together; 0 = no bound
    uint32_t route_cap = 0;  // nodes of the longest possible route
    uint64_t clock_ms = 0;   // end of the last tick
    uint64_t jobs = 0, completed = 0, rejected = 0;
    std::string err;
};

namespace {

int sfail(gmp_server* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

void release(gmp_server* s) {
    for (Slot& sl : s->slots)
        if (sl.ctx) gmp_destroy(sl.ctx);  // views: free their workspaces only
    s->slots.clear();
    if (s->state[1]) gmp_destroy(s->state[1]);
    s->state[1] = nullptr;
    for (cudaEvent_t& e : s->ready)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
}

uint64_t held_by_slots(const gmp_server* s) {
    uint64_t sum = 0;
    for (const Slot& sl : s->slots) sum += ctx_info(sl.ctx).used;
    return sum;
}

// Every request of a job that failed as a whole completes with the error.
void fail_job(gmp_server* s, uint32_t k, const std::vector<Request>& job, int rc) {
    const uint64_t t = now_ns();
    for (const Request& r : job) {
        Done d{};
        d.s.tag = r.tag;
        d.s.t_submit_ns = r.t_submit;
        d.s.t_launch_ns = t;
        d.s.t_done_ns = t;
        d.s.clock_ms = s->clock_ms;
        d.s.slot = k;
        d.s.batch_size = (uint32_t)job.size();
        d.s.result.status = rc;
        s->done.push_back(std::move(d));
    }
    s->completed += job.size();
}

// Admission: the number of requests at the head of the queue whose job fits the memory budget and the
// GPU's free memory on slot k (0: none fits right now).
uint32_t admit(gmp_server* s, uint32_t k) {
    gmp_ctx* c = s->slots[k].ctx;
    const uint64_t held = ctx_info(c).used;
    const uint64_t others = held_by_slots(s) - held;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    uint32_t n = (uint32_t)std::min<size_t>(s->cfg.max_batch, s->queue.size());
    while (n >= 1) {
        uint64_t ants = 0;
        uint32_t maxI = 1;
        for (uint32_t i = 0; i < n; ++i) {
            ants += s->queue[i].q.n_ants;
            maxI = std::max(maxI, s->queue[i].q.n_iter);
        }
        const uint64_t need = ctx_job_bytes(c, n, ants, maxI);  // what the slot would hold
        const uint64_t grow = need > held ? need - held : 0;
        const bool in_budget = !s->budget || others + need <= s->budget;
        // leave a small margin of the free memory for the allocator's own rounding
        if (need != ~0ull && in_budget && grow + (grow >> 4) <= (uint64_t)free_b) return n;
        n = n > 1 ? n - std::max<uint32_t>(1u, n / 4u) : 0u;
    }
    return 0;
}

// Launch a job on an idle slot from the head of the queue.
int launch_slot(gmp_server* s, uint32_t k) {
    Slot& sl = s->slots[k];
    uint32_t n = admit(s, k);
    if (n == 0) {
        bool any_busy = false;
        for (const Slot& o : s->slots) any_busy |= o.busy;
        if (any_busy) return GMP_OK;  // memory frees up as running jobs finish
        // nothing runs and not even one request fits: that request cannot be served
        std::vector<Request> one(1, s->queue.front());
        s->queue.pop_front();
        fail_job(s, k, one, GMP_ERR_OOM);
        return GMP_OK;
    }
    sl.job.assign(s->queue.begin(), s->queue.begin() + n);
    s->queue.erase(s->queue.begin(), s->queue.begin() + n);
    std::vector<gmp_query> qs(n);
    for (uint32_t i = 0; i < n; ++i) qs[i] = sl.job[i].q;
    // the job reads the current traffic-state version, after the tick that produced it, and departs at
    // the clock of that state
    const uint32_t v = s->cur;
    int rc = ctx_rebind_state(sl.ctx, s->state[v]);
    const CtxInfo ci = ctx_info(sl.ctx);
    if (rc == GMP_OK && s->has_ready[v] && cudaStreamWaitEvent(ci.stream, s->ready[v], 0) != cudaSuccess) {
        cudaGetLastError();
        rc = GMP_ERR_CUDA;
    }
    gmp_params p{};
    gmp_get_params(sl.ctx, &p);
    if (rc == GMP_OK && p.t_dep_ms != (uint32_t)s->clock_ms) {
        p.t_dep_ms = (uint32_t)s->clock_ms;
        rc = gmp_set_params(sl.ctx, &p);
    }
    if (rc == GMP_OK) rc = gmp_batch_stage(sl.ctx, n, qs.data());
    if (rc == GMP_OK) rc = gmp_batch_launch(sl.ctx);
    if (rc != GMP_OK) {
        bool any_busy = false;
        for (const Slot& o : s->slots) any_busy |= o.busy;
        if (rc == GMP_ERR_OOM && any_busy) {  // the allocator disagreed with the estimate: retry later
            s->queue.insert(s->queue.begin(), sl.job.begin(), sl.job.end());
            sl.job.clear();
            return GMP_OK;
        }
        fail_job(s, k, sl.job, rc);
        sl.job.clear();
        return GMP_OK;
    }
    sl.busy = true;
    sl.version = v;
    sl.t_launch = now_ns();
    sl.clock_ms = s->clock_ms;
    ++s->jobs;
    return GMP_OK;
}

// Collect a finished job into the completion queue.
int finish_slot(gmp_server* s, uint32_t k) {
    Slot& sl = s->slots[k];
    const uint64_t t_done = now_ns();
    const uint32_t n = (uint32_t)sl.job.size();
    sl.routes.resize((size_t)n * s->route_cap);
    sl.res.assign(n, gmp_result{});
    for (uint32_t i = 0; i < n; ++i) {
        sl.res[i].route = sl.routes.data() + (size_t)i * s->route_cap;
        sl.res[i].route_cap = s->route_cap;
    }
    const int rc = gmp_batch_collect(sl.ctx, sl.res.data());
    for (uint32_t i = 0; i < n; ++i) {
        Done d{};
        d.s.tag = sl.job[i].tag;
        d.s.t_submit_ns = sl.job[i].t_submit;
        d.s.t_launch_ns = sl.t_launch;
        d.s.t_done_ns = t_done;
        d.s.clock_ms = sl.clock_ms;
        d.s.slot = k;
        d.s.batch_size = n;
        d.s.result = sl.res[i];
        d.s.result.route = nullptr;
        d.s.result.route_cap = 0;
        if (rc != GMP_OK) {
            d.s.result.status = rc;
        } else if (sl.res[i].status == GMP_OK) {
            d.route.assign(sl.res[i].route, sl.res[i].route + sl.res[i].route_len);
        }
        s->done.push_back(std::move(d));
    }
    s->completed += n;
    sl.job.clear();
    sl.busy = false;
    return GMP_OK;
}

}  // namespace

extern "C" {

int gmp_server_create(gmp_server** out, gmp_ctx* graph, uint32_t n_slots, const gmp_server_config* cfg) {
    if (!out || !graph || !cfg || n_slots == 0) return GMP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_batch == 0 || cfg->max_ants == 0 || cfg->max_iter == 0) return GMP_ERR_INVALID_ARG;
    const CtxInfo gi = ctx_info(graph);
    if (!gi.has_graph) return ctx_fail(graph, GMP_ERR_STATE, "the server needs the road graph loaded");
    if (!ctx_owns_state(graph)) return ctx_fail(graph, GMP_ERR_STATE, "the server's context must own its traffic state");
    gmp_params gp{};
    gmp_get_params(graph, &gp);
    gmp_server* s = new gmp_server();
    s->cfg = *cfg;
    s->budget = (uint64_t)cfg->mem_budget_mib << 20;
    s->state[0] = graph;
    const uint32_t max_steps = gp.max_steps ? gp.max_steps : std::min<uint32_t>(2u * (gi.N - 1u), 4096u);
    s->route_cap = std::min<uint32_t>(gi.N, std::max<uint32_t>(max_steps, 1u) + 1u);
    auto fail_create = [&](int rc, gmp_ctx* blame) {
        if (blame) ctx_fail(graph, rc, gmp_last_error(blame));
        release(s);
        delete s;
        return rc;
    };
    int rc = gmp_create(&s->state[1], gi.device, 0, nullptr);
    if (rc != GMP_OK) return fail_create(rc, nullptr);
    rc = gmp_share_graph(s->state[1], graph, 1);
    if (rc == GMP_OK) rc = gmp_set_params(s->state[1], &gp);
    if (rc != GMP_OK) return fail_create(rc, s->state[1]);
    for (cudaEvent_t& e : s->ready)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail_create(GMP_ERR_CUDA, nullptr);
        }
    for (uint32_t k = 0; k < n_slots; ++k) {
        Slot sl;
        rc = gmp_create(&sl.ctx, gi.device, 0, nullptr);
        if (rc != GMP_OK) return fail_create(rc, nullptr);
        s->slots.push_back(sl);
        ctx_set_stream_alloc(sl.ctx);
        rc = gmp_share_graph(sl.ctx, graph, 0);
        if (rc == GMP_OK) rc = gmp_set_params(sl.ctx, &gp);
        if (rc != GMP_OK) return fail_create(rc, sl.ctx);
    }
    *out = s;
    return GMP_OK;
}

void gmp_server_destroy(gmp_server* s) {
    if (!s) return;
    release(s);
    delete s;
}

const char* gmp_server_last_error(const gmp_server* s) { return s ? s->err.c_str() : "null server"; }

int gmp_server_memory(const gmp_server* s, uint64_t* slots_bytes, uint64_t* budget_bytes) {
    if (!s) return GMP_ERR_INVALID_ARG;
    if (slots_bytes) *slots_bytes = held_by_slots(s);
    if (budget_bytes) *budget_bytes = s->budget;
    return GMP_OK;
}

int gmp_server_submit(gmp_server* s, const gmp_query* q, uint64_t tag) {
    if (!s || !q) return GMP_ERR_INVALID_ARG;
    if (q->n_ants > s->cfg.max_ants || q->n_iter > s->cfg.max_iter) {
        ++s->rejected;
        return sfail(s, GMP_ERR_INVALID_ARG, "request exceeds the server's max_ants or max_iter");
    }
    const int rc = ctx_check_query(s->slots[0].ctx, *q);
    if (rc != GMP_OK) {
        ++s->rejected;
        return sfail(s, rc, gmp_last_error(s->slots[0].ctx));
    }
    s->queue.push_back(Request{*q, tag, now_ns()});
    return GMP_OK;
}

int gmp_server_tick(gmp_server* s, uint64_t t_now_ms, uint32_t dt_ms) {
    if (!s) return GMP_ERR_INVALID_ARG;
    if (t_now_ms + dt_ms >= (1ull << 30))
        return sfail(s, GMP_ERR_INVALID_ARG, "the serving clock (departure time) must stay below 2^30 ms");
    const uint32_t nx = s->cur ^ 1u;
    gmp_ctx* next = s->state[nx];
    cudaStream_t st = ctx_info(next).stream;
    // the version about to be overwritten: after every job still reading it; the version copied: after
    // the tick that produced it
    for (const Slot& sl : s->slots)
        if (sl.busy && sl.version == nx) {
            const cudaEvent_t e = ctx_done_event(sl.ctx);
            if (e && cudaStreamWaitEvent(st, e, 0) != cudaSuccess) {
                cudaGetLastError();
                return sfail(s, GMP_ERR_CUDA, "ordering the tick after running jobs failed");
            }
        }
    if (s->has_ready[s->cur] && cudaStreamWaitEvent(st, s->ready[s->cur], 0) != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, GMP_ERR_CUDA, "ordering the tick after the previous one failed");
    }
    int rc = ctx_copy_state(next, s->state[s->cur]);
    if (rc == GMP_OK) rc = gmp_tick(next, t_now_ms, dt_ms);
    if (rc != GMP_OK) return sfail(s, rc, gmp_last_error(next));
    if (cudaEventRecord(s->ready[nx], st) != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, GMP_ERR_CUDA, "recording the tick failed");
    }
    s->has_ready[nx] = true;
    s->cur = nx;
    s->clock_ms = t_now_ms + dt_ms;
    return GMP_OK;
}

int gmp_server_pump(gmp_server* s, gmp_server_stats* st) {
    if (!s) return GMP_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < s->slots.size(); ++k) {
        Slot& sl = s->slots[k];
        if (!sl.busy) continue;
        int ready = 0;
        int rc = gmp_batch_ready(sl.ctx, &ready);
        if (rc != GMP_OK || ready) rc = finish_slot(s, k);
        if (rc != GMP_OK) return sfail(s, rc, gmp_last_error(sl.ctx));
    }
    for (uint32_t k = 0; k < s->slots.size() && !s->queue.empty(); ++k)
        if (!s->slots[k].busy) {
            const int rc = launch_slot(s, k);
            if (rc != GMP_OK) return rc;
        }
    if (st) {
        memset(st, 0, sizeof *st);
        st->queued = (uint32_t)s->queue.size();
        for (const Slot& sl : s->slots) {
            st->busy_slots += sl.busy ? 1u : 0u;
            st->in_flight += (uint32_t)sl.job.size();
        }
        st->done_waiting = (uint32_t)s->done.size();
        st->jobs = s->jobs;
        st->completed = s->completed;
        st->rejected = s->rejected;
    }
    return GMP_OK;
}

int gmp_server_take(gmp_server* s, uint32_t max_n, gmp_served* out, uint32_t* route_buf, uint64_t route_entries,
                    uint32_t* n_out) {
    if (!s || !n_out || (max_n && !out)) return GMP_ERR_INVALID_ARG;
    uint32_t n = 0;
    uint64_t used = 0;
    while (n < max_n && !s->done.empty()) {
        Done& d = s->done.front();
        const uint64_t len = d.route.size();
        if (len && (!route_buf || used + len > route_entries)) {
            if (n == 0) {
                *n_out = 0;
                return sfail(s, GMP_ERR_BUFFER, "route buffer too small for the next result");
            }
            break;
        }
        out[n] = d.s;
        if (len) {
            memcpy(route_buf + used, d.route.data(), len * 4);
            out[n].result.route = route_buf + used;
            out[n].result.route_cap = (uint32_t)len;
            used += len;
        }
        s->done.pop_front();
        ++n;
    }
    *n_out = n;
    return GMP_OK;
}

}  // extern "C"

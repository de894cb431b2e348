// Route server with continuous batching (gmp_server_*, declared in include/gmacop.h).
//
// The paper routes vehicles one request at a time (Fig. 3); a deployment receives route requests
// continuously while the traffic state changes. The server keeps that state resident on the device
// and runs colonies as they arrive:
//   - slots: each slot is a context holding its own replica of the road graph, signals and traffic
//     state, on its own CUDA stream, so jobs of different slots overlap on the GPU and never share a
//     buffer another job writes;
//   - admission by memory: each slot reserves, once, the workspace of its largest job; the number of
//     requests a job may hold is what the slot's memory budget admits (up to max_batch);
//   - continuous batching: whenever a slot is idle, everything waiting (up to that capacity) becomes
//     the slot's next job, launched without waiting for any other slot;
//   - ticks: a traffic tick is issued on every slot's stream, so it lands between that slot's jobs;
//     each request departs at, and records, the traffic clock of the state it was solved on.
// A request's result depends only on the request and that state (Philox streams are keyed by the
// request's own seed), so it is the same alone and in any mix. The server is single-threaded: the
// caller drives it with gmp_server_pump.
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
    gmp_ctx* ctx = nullptr;
    uint32_t cap = 0;  // requests per job the slot's memory admits
    bool busy = false;
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
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::deque<Done> done;
    gmp_server_config cfg{};
    uint32_t route_cap = 0;  // max_steps + 1 of the graph
    uint64_t clock_ms = 0;   // end of the last tick
    uint64_t jobs = 0, completed = 0, rejected = 0;
    std::string err;
};

namespace {

int sfail(gmp_server* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

// Launch a job on an idle slot from the head of the queue.
int launch_slot(gmp_server* s, uint32_t k) {
    Slot& sl = s->slots[k];
    const uint32_t n = (uint32_t)std::min<size_t>(sl.cap, s->queue.size());
    if (n == 0) return GMP_OK;
    sl.job.assign(s->queue.begin(), s->queue.begin() + n);
    s->queue.erase(s->queue.begin(), s->queue.begin() + n);
    std::vector<gmp_query> qs(n);
    for (uint32_t i = 0; i < n; ++i) qs[i] = sl.job[i].q;
    // the job departs at the traffic clock of the state it runs on
    gmp_params p{};
    gmp_get_params(sl.ctx, &p);
    int rc = GMP_OK;
    if (p.t_dep_ms != (uint32_t)s->clock_ms) {
        p.t_dep_ms = (uint32_t)s->clock_ms;
        rc = gmp_set_params(sl.ctx, &p);
    }
    if (rc == GMP_OK) rc = gmp_batch_stage(sl.ctx, n, qs.data());
    if (rc == GMP_OK) rc = gmp_batch_launch(sl.ctx);
    if (rc != GMP_OK) {  // the whole job fails: every request completes with the error
        const uint64_t t = now_ns();
        for (const Request& r : sl.job) {
            Done d{};
            d.s.tag = r.tag;
            d.s.t_submit_ns = r.t_submit;
            d.s.t_launch_ns = t;
            d.s.t_done_ns = t;
            d.s.clock_ms = s->clock_ms;
            d.s.slot = k;
            d.s.batch_size = n;
            d.s.result.status = rc;
            s->done.push_back(std::move(d));
        }
        s->completed += n;
        sl.job.clear();
        return GMP_OK;
    }
    sl.busy = true;
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

int gmp_server_create(gmp_server** out, gmp_ctx* const* slots, uint32_t n_slots, const gmp_server_config* cfg) {
    if (!out || !slots || !cfg || n_slots == 0) return GMP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_batch == 0 || cfg->max_ants == 0 || cfg->max_iter == 0) return GMP_ERR_INVALID_ARG;
    gmp_server* s = new gmp_server();
    s->cfg = *cfg;
    uint32_t N = 0, E = 0;
    for (uint32_t k = 0; k < n_slots; ++k) {
        if (!slots[k]) {
            delete s;
            return GMP_ERR_INVALID_ARG;
        }
        const CtxInfo ci = ctx_info(slots[k]);
        if (!ci.has_graph) {
            delete s;
            return ctx_fail(slots[k], GMP_ERR_STATE, "every slot needs the road graph loaded");
        }
        if (k > 0 && (ci.N != N || ci.E != E)) {
            delete s;
            return ctx_fail(slots[k], GMP_ERR_INVALID_ARG, "slots must hold the same road graph");
        }
        N = ci.N;
        E = ci.E;
        gmp_params p{};
        gmp_get_params(slots[k], &p);
        const uint32_t max_steps = p.max_steps ? p.max_steps : std::min<uint32_t>(N > 0 ? N - 1 : 0, 4096u);
        s->route_cap = std::max<uint32_t>(max_steps, 1u) + 1u;
        // admission by memory: the largest job this slot's budget holds, up to max_batch requests
        uint32_t cap = cfg->max_batch;
        int rc = GMP_ERR_OOM;
        while (cap >= 1) {
            rc = gmp_batch_reserve(slots[k], cap, (uint64_t)cap * cfg->max_ants, cfg->max_iter);
            if (rc != GMP_ERR_OOM) break;
            cap = cap > 1 ? cap - std::max<uint32_t>(1u, cap / 4u) : 0u;
        }
        if (rc != GMP_OK) {
            delete s;
            return rc;
        }
        Slot sl;
        sl.ctx = slots[k];
        sl.cap = cap;
        s->slots.push_back(std::move(sl));
    }
    *out = s;
    return GMP_OK;
}

void gmp_server_destroy(gmp_server* s) { delete s; }

const char* gmp_server_last_error(const gmp_server* s) { return s ? s->err.c_str() : "null server"; }

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
    for (Slot& sl : s->slots) {
        const int rc = gmp_tick(sl.ctx, t_now_ms, dt_ms);
        if (rc != GMP_OK) return sfail(s, rc, gmp_last_error(sl.ctx));
    }
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

int gmp_server_slot_capacity(const gmp_server* s, uint32_t slot, uint32_t* requests_per_job) {
    if (!s || !requests_per_job || slot >= s->slots.size()) return GMP_ERR_INVALID_ARG;
    *requests_per_job = s->slots[slot].cap;
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

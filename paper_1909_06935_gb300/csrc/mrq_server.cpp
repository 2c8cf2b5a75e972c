// mrq_server.cpp - request server over the C ABI (continuous batching of sampling requests).
//
// Requests (a Hamiltonian, a reference, sampling coefficients, sampling parameters, a target
// error and a step limit) wait in a FIFO queue.  Each scheduling round:
//   1. admits queued requests while the device-memory budget and the active-slot limit allow
//      (each admitted request gets its own context: integrals, hash table, coefficients and
//      walkers stay resident until it retires),
//   2. advances the walkers of every active request together (mrq_batch_advance: one walk
//      launch per determinant width),
//   3. finalizes every active request and retires those that reached their target sigma of
//      E^(2) (after the burn-in) or their step limit, freeing their device memory.
// A request's walkers advance by the same steps whatever else is active, so its trajectory is the
// same alone and in the mix.  The paper runs one system per job; this is the serving form.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mrq.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    // owned copies of the inputs
    int n_core = 0, n_act = 0, n_virt = 0, n_alpha = 0, n_beta = 0;
    double e_core = 0.0;
    std::vector<double> h1, eri, coeffs, c;
    std::vector<uint64_t> dets;
    mrq_sample_params params{};
    double target_sigma = 0.0;
    int64_t max_steps = 0;
    // state
    int state = MRQ_REQ_QUEUED;
    int status = 0;
    int64_t steps_done = 0;
    int64_t footprint = 0;
    mrq_ctx* ctx = nullptr;
    mrq_result result{};
    clk::time_point t_submit, t_admit, t_done;
};

int64_t nsub2(int64_t k) { return k * (k - 1) / 2; }

// device bytes a request keeps resident while active (integral tables, hash, coefficients,
// accumulators, walkers, candidate scratch) - an estimate used for admission
int64_t footprint_of(const Request& r) {
    const int64_t n = r.n_core + r.n_act + r.n_virt;
    const int64_t npair = n * (n + 1) / 2;
    const int64_t neri = npair * (npair + 1) / 2;
    const int64_t nlab = (1 + 2 * (int64_t)r.n_core + nsub2(2 * r.n_core)) *
                         (1 + 2 * (int64_t)r.n_virt + nsub2(2 * r.n_virt));
    int64_t cap = 16;
    while (cap < 4 * (int64_t)r.coeffs.size()) cap <<= 1;
    const int64_t G = std::max<int32_t>(r.params.n_groups, 1);
    int64_t b = 0;
    const int64_t nca = r.n_core + r.n_act, nav = r.n_act + r.n_virt;
    b += 8 * (2 * n * n + neri + npair * n * n + 2 * nca * nca * nav * nav + n + r.n_act * r.n_act);
    b += 16 * cap + 8 * nlab;
    b += 32 * G * nlab + 16 * G;        // N, U and the SC-MRCI gradient sums A, B per group
    b += 112 * r.params.n_walkers;     // walkers with their step records
    int64_t npad = 1;
    while (npad < r.params.n_walkers) npad <<= 1;
    b += 12 * npad;                     // slot ordering keys and indices
    b += 8 * (G + 1) * ((nlab + 8191) / 8192) * 45;   // finalize partial sums
    return b;
}

}  // namespace

struct mrq_server {
    mrq_server_params p{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::map<int64_t, Request*> all;
    int64_t next_ticket = 1;
    int64_t used_bytes = 0;
    std::thread worker;
    std::atomic<bool> stop{false};
    bool running = false;
    char err[512] = {0};
    int64_t rounds = 0, total_walker_steps = 0;
};

static void retire_locked(mrq_server* s, Request* r, int state) {
    if (r->ctx) {
        mrq_destroy(r->ctx);
        r->ctx = nullptr;
        s->used_bytes -= r->footprint;
    }
    r->state = state;
    r->t_done = clk::now();
    r->h1.clear();
    r->h1.shrink_to_fit();
    r->eri.clear();
    r->eri.shrink_to_fit();
    r->dets.clear();
    r->dets.shrink_to_fit();
    r->coeffs.clear();
    r->coeffs.shrink_to_fit();
    r->c.clear();
    r->c.shrink_to_fit();
}

// load a queued request onto the device (called with the lock released)
static int admit(mrq_server* s, Request* r) {
    mrq_ctx* ctx = nullptr;
    int rc = mrq_create(&ctx, s->p.device);
    if (rc) return rc;
    rc = mrq_load_hamiltonian(ctx, r->n_core, r->n_act, r->n_virt, r->n_alpha, r->n_beta, r->h1.data(), r->eri.data(),
                              r->e_core);
    if (!rc) rc = mrq_load_reference(ctx, (int64_t)r->coeffs.size(), r->dets.data(), r->coeffs.data());
    if (!rc && !r->c.empty()) rc = mrq_set_coeffs(ctx, (int64_t)r->c.size(), r->c.data());
    if (!rc) {
        mrq_sample_params q = r->params;
        q.n_steps = 0;
        rc = mrq_walkers_init(ctx, &q);
    }
    if (rc) {
        snprintf(s->err, sizeof s->err, "ticket %lld: %s", (long long)r->ticket, mrq_last_error(ctx));
        mrq_destroy(ctx);
        return rc;
    }
    r->ctx = ctx;
    return 0;
}

static int server_round(mrq_server* s) {
    // 1. admission (FIFO; stop at the first request that does not fit)
    for (;;) {
        Request* r = nullptr;
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->queue.empty() || (int)s->active.size() >= s->p.max_active) break;
            Request* head = s->queue.front();
            if (head->state == MRQ_REQ_CANCELLED) {
                s->queue.pop_front();
                continue;
            }
            if (s->used_bytes + head->footprint > s->p.hbm_budget_bytes && !s->active.empty()) break;
            s->queue.pop_front();
            r = head;
            s->used_bytes += r->footprint;
        }
        const int rc = admit(s, r);
        std::lock_guard<std::mutex> g(s->mu);
        if (rc) {
            r->status = rc;
            s->used_bytes -= r->footprint;
            retire_locked(s, r, MRQ_REQ_FAILED);
        } else {
            r->state = MRQ_REQ_RUNNING;
            r->t_admit = clk::now();
            s->active.push_back(r);
        }
    }
    // 2. one batched advance of every active request
    std::vector<Request*> act;
    {
        std::lock_guard<std::mutex> g(s->mu);
        for (Request* r : s->active)
            if (r->state == MRQ_REQ_RUNNING) act.push_back(r);
    }
    if (act.empty()) return 0;
    std::vector<mrq_ctx*> ctxs;
    for (Request* r : act) ctxs.push_back(r->ctx);
    const int64_t steps = s->p.steps_per_round;
    int rc = mrq_batch_advance(ctxs.data(), (int)ctxs.size(), steps);
    if (rc) snprintf(s->err, sizeof s->err, "batched advance failed: %s", mrq_last_error(ctxs[0]));
    // 3. finalize with the lock released (only this thread uses an active request's context, and
    //    only this thread retires running requests), then retire under the lock
    std::vector<mrq_result> res(act.size());
    std::vector<int> fr(act.size(), 0);
    if (!rc)
        for (size_t i = 0; i < act.size(); i++) fr[i] = mrq_finalize(act[i]->ctx, &res[i]);
    std::lock_guard<std::mutex> g(s->mu);
    s->rounds++;
    std::vector<Request*> keep;
    for (Request* r : s->active) {
        if (r->state == MRQ_REQ_CANCELLED) {
            retire_locked(s, r, MRQ_REQ_CANCELLED);
            continue;
        }
        const size_t i = (size_t)(std::find(act.begin(), act.end(), r) - act.begin());
        if (i == act.size()) {          // admitted after the snapshot: nothing ran yet
            keep.push_back(r);
            continue;
        }
        if (rc) {
            r->status = rc;
            retire_locked(s, r, MRQ_REQ_FAILED);
            continue;
        }
        r->steps_done += steps;
        s->total_walker_steps += steps * r->params.n_walkers;
        r->result = res[i];
        if (fr[i]) {
            r->status = fr[i];
            retire_locked(s, r, MRQ_REQ_FAILED);
            continue;
        }
        const bool converged = r->target_sigma > 0.0 && r->steps_done > r->params.burn_in &&
                               res[i].walker_steps > 0 && res[i].e2_sigma <= r->target_sigma;
        if (converged || r->steps_done >= r->max_steps) retire_locked(s, r, MRQ_REQ_DONE);
        else keep.push_back(r);
    }
    s->active.swap(keep);
    s->cv.notify_all();
    return rc;
}

extern "C" {

int mrq_server_create(mrq_server** out, const mrq_server_params* p) {
    if (!out || !p || p->max_active <= 0 || p->steps_per_round <= 0 || p->hbm_budget_bytes <= 0)
        return MRQ_INVALID_ARG;
    mrq_server* s = new mrq_server();
    s->p = *p;
    *out = s;
    return 0;
}

int mrq_server_submit(mrq_server* s, const mrq_request* q, int64_t* ticket) {
    if (!s || !q || !ticket || !q->h1 || !q->eri || !q->dets || !q->coeffs || q->n_det <= 0) return MRQ_INVALID_ARG;
    const int n = q->n_core + q->n_act + q->n_virt;
    if (n <= 0 || n > 128 || q->params.n_walkers <= 0 || q->max_steps <= 0) return MRQ_INVALID_ARG;
    Request* r = new Request();
    r->n_core = q->n_core;
    r->n_act = q->n_act;
    r->n_virt = q->n_virt;
    r->n_alpha = q->n_alpha;
    r->n_beta = q->n_beta;
    r->e_core = q->e_core;
    const int64_t npair = (int64_t)n * (n + 1) / 2;
    const int W = (n + 63) / 64;
    r->h1.assign(q->h1, q->h1 + (size_t)n * n);
    r->eri.assign(q->eri, q->eri + (size_t)(npair * (npair + 1) / 2));
    r->dets.assign(q->dets, q->dets + (size_t)q->n_det * 2 * W);
    r->coeffs.assign(q->coeffs, q->coeffs + (size_t)q->n_det);
    if (q->c && q->n_labels > 0) r->c.assign(q->c, q->c + (size_t)q->n_labels);
    r->params = q->params;
    r->target_sigma = q->target_sigma;
    r->max_steps = q->max_steps;
    r->footprint = footprint_of(*r);
    r->t_submit = clk::now();
    std::lock_guard<std::mutex> g(s->mu);
    if (r->footprint > s->p.hbm_budget_bytes) {
        r->state = MRQ_REQ_FAILED;
        r->status = MRQ_TOO_LARGE;
    }
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    if (r->state == MRQ_REQ_QUEUED) s->queue.push_back(r);
    else r->t_done = r->t_submit;
    *ticket = r->ticket;
    s->cv.notify_all();
    return 0;
}

int mrq_server_poll(mrq_server* s, int64_t ticket, mrq_request_status* out) {
    if (!s || !out) return MRQ_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return MRQ_INVALID_ARG;
    const Request* r = it->second;
    out->state = r->state;
    out->status = r->status;
    out->steps_done = r->steps_done;
    out->result = r->result;
    auto secs = [](clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); };
    const bool finished = r->state == MRQ_REQ_DONE || r->state == MRQ_REQ_FAILED || r->state == MRQ_REQ_CANCELLED;
    out->queue_seconds = r->state == MRQ_REQ_QUEUED ? secs(r->t_submit, clk::now())
                                                    : (r->ctx || finished) && r->t_admit.time_since_epoch().count()
                                                          ? secs(r->t_submit, r->t_admit)
                                                          : 0.0;
    out->total_seconds = finished ? secs(r->t_submit, r->t_done) : secs(r->t_submit, clk::now());
    return 0;
}

int mrq_server_cancel(mrq_server* s, int64_t ticket) {
    if (!s) return MRQ_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return MRQ_INVALID_ARG;
    Request* r = it->second;
    if (r->state == MRQ_REQ_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
        retire_locked(s, r, MRQ_REQ_CANCELLED);
    } else if (r->state == MRQ_REQ_RUNNING) {
        r->state = MRQ_REQ_CANCELLED;     // retired at the end of the current round
    }
    return 0;
}

int mrq_server_step(mrq_server* s) {
    if (!s) return MRQ_INVALID_ARG;
    if (s->running) return MRQ_INVALID_ARG;   // the background loop owns the rounds
    return server_round(s);
}

int mrq_server_start(mrq_server* s) {
    if (!s || s->running) return MRQ_INVALID_ARG;
    s->stop = false;
    s->running = true;
    s->worker = std::thread([s]() {
        while (!s->stop.load()) {
            bool idle;
            {
                std::unique_lock<std::mutex> g(s->mu);
                idle = s->queue.empty() && s->active.empty();
                if (idle) s->cv.wait_for(g, std::chrono::milliseconds(2));
            }
            if (!idle) server_round(s);
        }
    });
    return 0;
}

int mrq_server_stop(mrq_server* s) {
    if (!s) return MRQ_INVALID_ARG;
    if (s->running) {
        s->stop = true;
        s->cv.notify_all();
        s->worker.join();
        s->running = false;
    }
    return 0;
}

int mrq_server_info(mrq_server* s, int64_t* out4) {
    if (!s || !out4) return MRQ_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    out4[0] = (int64_t)s->queue.size();
    out4[1] = (int64_t)s->active.size();
    out4[2] = s->used_bytes;
    out4[3] = s->total_walker_steps;
    return 0;
}

const char* mrq_server_last_error(const mrq_server* s) { return s ? s->err : "null server"; }

void mrq_server_destroy(mrq_server* s) {
    if (!s) return;
    mrq_server_stop(s);
    std::lock_guard<std::mutex> g(s->mu);
    for (auto& kv : s->all) {
        Request* r = kv.second;
        if (r->ctx) mrq_destroy(r->ctx);
        delete r;
    }
    delete s;
}

}  // extern "C"

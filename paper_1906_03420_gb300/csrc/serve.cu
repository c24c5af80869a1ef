// Batched and served execution (host side).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "common.cuh"
#include "internal.h"
#include "runtime.h"

using namespace gsi;

extern "C" gsi_status gsi_batch_run(gsi_graph *g, const gsi_query_desc *qs, int32_t nq, const gsi_batch_opts *opts,
                                    gsi_result **outs, int32_t *statuses) {
    if (!g || (nq > 0 && (!qs || !outs)) || nq < 0) {
        set_error("gsi_batch_run: null argument");
        return GSI_EINVAL;
    }
    gsi_batch_opts bo;
    std::memset(&bo, 0, sizeof bo);
    if (opts) bo = *opts;
    gsi_status first_err = GSI_OK;
    for (int32_t i = 0; i < nq; ++i) {
        outs[i] = nullptr;
        QueryGraph q;
        gsi_status rc = validate_query(qs[i].vlab, qs[i].k, qs[i].src, qs[i].dst, qs[i].elab, qs[i].qm, &q);
        if (rc == GSI_OK) {
            gsi_query_opts o;
            std::memset(&o, 0, sizeof o);
            o.stream = bo.stream;
            o.row_cap = bo.row_cap;
            o.mem_budget = bo.mem_budget;
            o.count_only = bo.count_only;
            o.stats = bo.stats;
            rc = run_query(g, q, o, &outs[i]);
        }
        if (statuses) statuses[i] = rc;
        if (rc != GSI_OK && first_err == GSI_OK && rc != GSI_EINVAL) first_err = rc;
    }
    return first_err;
}

// ------------------------------------------------------------------ server
struct gsi_server {
    gsi_graph *g = nullptr;
    gsi_server_opts opts;
    struct Req {
        uint64_t ticket;
        QueryGraph q;
        std::chrono::steady_clock::time_point t_submit;
        gsi_status status = GSI_EBUSY;
        gsi_result *res = nullptr;
        double latency_ms = 0;
        bool cancelled = false;
    };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::map<uint64_t, std::shared_ptr<Req>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
};

static void server_worker(gsi_server *s, int idx) {
    cudaSetDevice(s->g->device);
    cudaStream_t st = s->streams[idx];
    for (;;) {
        std::shared_ptr<gsi_server::Req> r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop && s->queue.empty()) return;
            r = s->queue.front();
            s->queue.pop_front();
            if (r->cancelled) {
                r->status = GSI_ECANCELLED;
                s->cv_done.notify_all();
                continue;
            }
        }
        gsi_query_opts o;
        std::memset(&o, 0, sizeof o);
        o.stream = st;
        o.row_cap = s->opts.row_cap;
        o.count_only = s->opts.count_only;
        o.mem_budget = s->opts.mem_budget / (uint64_t)std::max(1, s->opts.n_streams);
        gsi_result *res = nullptr;
        gsi_status rc = run_query(s->g, r->q, o, &res);
        auto now = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            r->res = res;
            r->status = rc;
            r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
        }
        s->cv_done.notify_all();
    }
}

extern "C" gsi_status gsi_server_create(gsi_graph *g, const gsi_server_opts *opts, gsi_server **out) {
    if (!g || !out) {
        set_error("gsi_server_create: null argument");
        return GSI_EINVAL;
    }
    GSI_TRY(prepare_device(g->device));
    std::unique_ptr<gsi_server> s(new gsi_server());
    s->g = g;
    std::memset(&s->opts, 0, sizeof s->opts);
    if (opts) s->opts = *opts;
    if (s->opts.n_streams < 1) s->opts.n_streams = 4;
    if (s->opts.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        GSI_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        s->opts.mem_budget = fr / 2;
    }
    for (int i = 0; i < s->opts.n_streams; ++i) {
        cudaStream_t st;
        GSI_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        s->streams.push_back(st);
    }
    for (int i = 0; i < s->opts.n_streams; ++i) s->workers.emplace_back(server_worker, s.get(), i);
    *out = s.release();
    return GSI_OK;
}

extern "C" gsi_status gsi_server_submit(gsi_server *s, const gsi_query_desc *q, uint64_t *ticket) {
    if (!s || !q || !ticket) {
        set_error("gsi_server_submit: null argument");
        return GSI_EINVAL;
    }
    auto r = std::make_shared<gsi_server::Req>();
    GSI_TRY(validate_query(q->vlab, q->k, q->src, q->dst, q->elab, q->qm, &r->q));
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return GSI_OK;
}

extern "C" gsi_status gsi_server_poll(gsi_server *s, uint64_t ticket, int32_t timeout_ms, gsi_result **out,
                                      double *latency_ms) {
    if (!s || !out) {
        set_error("gsi_server_poll: null argument");
        return GSI_EINVAL;
    }
    *out = nullptr;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("gsi_server_poll: unknown ticket");
        return GSI_EINVAL;
    }
    auto r = it->second;
    auto done = [&] { return r->status != GSI_EBUSY; };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    if (!done()) return GSI_EBUSY;
    s->all.erase(it);
    if (latency_ms) *latency_ms = r->latency_ms;
    if (r->status != GSI_OK) {
        set_error("gsi_server_poll: query failed");
        return r->status;
    }
    *out = r->res;
    return GSI_OK;
}

extern "C" gsi_status gsi_server_cancel(gsi_server *s, uint64_t ticket) {
    if (!s) {
        set_error("gsi_server_cancel: null server");
        return GSI_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("gsi_server_cancel: unknown ticket");
        return GSI_EINVAL;
    }
    it->second->cancelled = true;
    return GSI_OK;
}

extern "C" void gsi_server_destroy(gsi_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &w : s->workers) w.join();
    for (auto &kv : s->all)
        if (kv.second->res) gsi_result_destroy(kv.second->res);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
}

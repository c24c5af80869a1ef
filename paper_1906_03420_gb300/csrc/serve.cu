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

// Batched queries (a shared work queue in one persistent launch, batch.cu):
// one filter launch per query, one readback of every |C(u)|, host plans, then
// the batch kernel.  Queries whose tables did not fit the batch arena run
// again on the plain path.
// Batched queries (a shared work queue in one persistent launch, batch.cu):
// one filter pass for every query vertex of the batch, one readback of every
// |C(u)|, host plans, then the batch kernel.  Queries whose tables did not fit
// the batch arena run again on the plain path.  Invalid queries carry their
// status in plans[i].status.
namespace gsi {
// The first half of a batch: queries that cannot match (a label no data
// vertex or edge carries) become inactive, one filter pass covers every query
// vertex of the rest, and each query with non-empty candidate sets gets its
// Alg. 2 order and steps.  The bitmaps stay allocated in `in` (the join reads
// them) until batch_inputs_free.
gsi_status batch_plan_all(gsi_graph *g, std::vector<BatchPlan> &plans, gsi_stats *stats, cudaStream_t st,
                          BatchInputs &in) {
    const int32_t nq = (int32_t)plans.size();
    std::vector<int32_t> ranks((size_t)nq * GSI_MAX_QUERY_VERTICES, 0);
    uint64_t bm_words = 0, nk = 0;
    std::vector<uint64_t> bm_off((size_t)nq, 0), k_off((size_t)nq, 0);
    for (int32_t i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        p.active = false;
        if (p.status != GSI_OK) continue;
        p.k = p.q.k;
        bool empty = (p.k > 1 && g->m == 0);
        for (int e = 0; e < p.q.qm && !empty; ++e) empty |= p.q.lab[e] >= g->L || g->freq[p.q.lab[e]] == 0;
        for (int u = 0; u < p.k && !empty; ++u) {
            ranks[(size_t)i * GSI_MAX_QUERY_VERTICES + u] = g->label_rank(p.q.vlab[u]);
            empty |= ranks[(size_t)i * GSI_MAX_QUERY_VERTICES + u] < 0;
        }
        if (empty) continue;
        p.active = true;
        bm_off[i] = bm_words;
        k_off[i] = nk;
        bm_words += (uint64_t)p.k * (uint64_t)g->nwords;
        nk += (uint64_t)p.k;
    }
    in.nk = nk;
    if (nk == 0) return GSI_OK;
    GSI_CUDA_TRY(cudaMallocAsync(&in.bitmaps, bm_words * 4 + 16, st));
    GSI_CUDA_TRY(cudaMallocAsync(&in.counts, nk * 8, st));
    std::vector<QuerySig> sigs;
    sigs.reserve((size_t)nq);
    for (int32_t i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        if (!p.active) continue;
        sigs.emplace_back();
        query_signatures(p.q.vl.data(), p.k, p.q.src.data(), p.q.dst.data(), p.q.lab.data(), p.q.qm, &sigs.back());
        p.bitmaps = in.bitmaps + bm_off[i];
        in.labels.insert(in.labels.end(), p.q.vlab, p.q.vlab + p.k);
    }
    std::vector<const uint32_t *> sp;
    for (const QuerySig &q : sigs)
        for (int u = 0; u < q.k; ++u) sp.push_back(q.sig[u]);
    GSI_TRY(filter_plan(g, sp, &in.fp, st));
    cudaEvent_t f0 = nullptr, f1 = nullptr;
    if (stats) {
        cudaEventCreate(&f0);
        cudaEventCreate(&f1);
        cudaEventRecord(f0, st);
    }
    gsi_status rc = filter_enqueue(g, in.fp, in.bitmaps, in.counts, st);
    if (stats) cudaEventRecord(f1, st);
    std::vector<uint64_t> hc(nk);
    if (rc == GSI_OK && (cudaMemcpyAsync(hc.data(), in.counts, nk * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess)) {
        set_error("batch: filter readback failed");
        rc = GSI_ECUDA;
    }
    if (stats) {
        float ms = 0;
        if (rc == GSI_OK) cudaEventElapsedTime(&ms, f0, f1);
        stats->filter_ms += ms;
        stats->filter_launches += 1;
        stats->kernels += 1;
        stats->filter_bytes += filter_alg_bytes(g, in.labels);
        cudaEventDestroy(f0);
        cudaEventDestroy(f1);
    }
    if (rc != GSI_OK) return rc;
    for (int32_t i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        if (!p.active) continue;
        const uint64_t *c = hc.data() + k_off[i];
        bool empty = false;
        for (int u = 0; u < p.k; ++u) empty |= c[u] == 0;
        if (empty) {
            p.active = false;
            continue;
        }
        plan_for_batch(g, p, c, ranks.data() + (size_t)i * GSI_MAX_QUERY_VERTICES);
    }
    return GSI_OK;
}

void batch_inputs_free(BatchInputs &in, cudaStream_t st) {
    if (in.bitmaps) cudaFreeAsync(in.bitmaps, st);
    if (in.counts) cudaFreeAsync(in.counts, st);
    filter_plan_free(in.fp, st);
    in = BatchInputs();
}

// The second half: a result object per query from its plan (rows in the
// batch's shared buffer), or a rerun on the plain path for a failed query.
gsi_status batch_finish(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &bo, uint64_t budget,
                        cudaStream_t st, std::vector<gsi_result *> &outs, std::vector<gsi_status> &statuses) {
    const int32_t nq = (int32_t)plans.size();
    outs.assign((size_t)nq, nullptr);
    statuses.assign((size_t)nq, GSI_OK);
    gsi_status first_err = GSI_OK;
    for (int32_t i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        gsi_status qrc = p.status;
        if (qrc == GSI_OK && p.active && p.failed) {
            gsi_query_opts o;
            std::memset(&o, 0, sizeof o);
            o.stream = st;
            o.row_cap = bo.row_cap;
            o.mem_budget = budget;
            o.count_only = bo.count_only;
            o.stats = bo.stats;
            qrc = run_query(g, p.q, o, &outs[i]);
            if (bo.stats) bo.stats->host_driven += 1;
        } else if (qrc == GSI_OK) {
            gsi_result *r = new gsi_result();
            r->k = p.k;
            r->device = g->device;
            r->stream = st;
            r->own_stream = true;
            r->count = p.active ? p.count : 0;
            uint64_t keep = bo.count_only ? 0 : (bo.row_cap ? bo.row_cap : UINT64_MAX);
            for (auto &c : p.chunks) {
                if (r->materialised >= keep) break;
                gsi_result::Chunk ch = c;
                ch.nrows = std::min<uint64_t>(ch.nrows, keep - r->materialised);
                ch.owned = false;                // rows live in the batch's shared buffer
                r->chunks.push_back(ch);
                r->materialised += ch.nrows;
            }
            r->arena = p.arena;
            outs[i] = r;
        }
        statuses[i] = qrc;
        if (qrc != GSI_OK && qrc != GSI_EINVAL && first_err == GSI_OK) first_err = qrc;
    }
    return first_err;
}

uint64_t batch_budget(const gsi_batch_opts &bo) {
    if (bo.mem_budget) return bo.mem_budget;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    return (uint64_t)(0.4 * (double)tot);
}

gsi_status batch_execute(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &bo,
                         std::vector<gsi_result *> &outs, std::vector<gsi_status> &statuses, BatchWorkspace *ws) {
    const int32_t nq = (int32_t)plans.size();
    outs.assign((size_t)nq, nullptr);
    statuses.assign((size_t)nq, GSI_OK);
    GSI_TRY(prepare_device(g->device));
    cudaStream_t st = (cudaStream_t)bo.stream;
    const uint64_t budget = batch_budget(bo);
    BatchInputs in;
    gsi_status rc = batch_plan_all(g, plans, bo.stats, st, in);
    if (rc == GSI_OK) rc = batch_run_device(g, plans, bo, budget, st, bo.stats, ws);
    batch_inputs_free(in, st);
    if (rc != GSI_OK) return rc;
    return batch_finish(g, plans, bo, budget, st, outs, statuses);
}
}  // namespace gsi

extern "C" gsi_status gsi_batch_run(gsi_graph *g, const gsi_query_desc *qs, int32_t nq, const gsi_batch_opts *opts,
                                    gsi_result **outs, int32_t *statuses) {
    if (!g || (nq > 0 && (!qs || !outs)) || nq < 0) {
        set_error("gsi_batch_run: null argument");
        return GSI_EINVAL;
    }
    try {
        gsi_batch_opts bo;
        std::memset(&bo, 0, sizeof bo);
        if (opts) bo = *opts;
        std::vector<BatchPlan> plans((size_t)nq);
        for (int32_t i = 0; i < nq; ++i)
            plans[i].status = validate_query(qs[i].vlab, qs[i].k, qs[i].src, qs[i].dst, qs[i].elab, qs[i].qm,
                                             &plans[i].q);
        std::vector<gsi_result *> res;
        std::vector<gsi_status> sts;
        gsi_status rc = batch_execute(g, plans, bo, res, sts);
        for (int32_t i = 0; i < nq; ++i) {
            outs[i] = i < (int32_t)res.size() ? res[i] : nullptr;
            if (statuses) statuses[i] = i < (int32_t)sts.size() ? sts[i] : rc;
        }
        return rc;
    } catch (const std::bad_alloc &) {
        set_error("gsi_batch_run: host allocation failed");
        return GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_batch_run: unexpected host exception");
        return GSI_ECUDA;
    }
}

extern "C" gsi_status gsi_batch_autotune(gsi_graph *g, const gsi_query_desc *qs, int32_t nq,
                                         const gsi_batch_opts *opts, int32_t *best_seeds_per_item,
                                         int32_t *best_item_rows, double *best_ms) {
    if (!g || nq < 1 || !qs) {
        set_error("gsi_batch_autotune: need a graph and at least one query");
        return GSI_EINVAL;
    }
    try {
        gsi_batch_opts bo;
        std::memset(&bo, 0, sizeof bo);
        if (opts) bo = *opts;
        bo.stats = nullptr;
        std::vector<BatchPlan> proto((size_t)nq);
        for (int32_t i = 0; i < nq; ++i)
            proto[i].status = validate_query(qs[i].vlab, qs[i].k, qs[i].src, qs[i].dst, qs[i].elab, qs[i].qm,
                                             &proto[i].q);
        const int32_t cand_spi[] = {32, 64, 128};
        const int32_t cand_rows[] = {512, 1024, 2048};
        double best = 1e300;
        int32_t arg_spi = 32, arg_rows = 1024;
        for (int32_t spi : cand_spi) {
            for (int32_t rows : cand_rows) {
                double t_best = 1e300;
                for (int rep = 0; rep < 2; ++rep) {
                    std::vector<BatchPlan> plans((size_t)nq);
                    for (int32_t i = 0; i < nq; ++i) {
                        plans[i].status = proto[i].status;
                        plans[i].q = proto[i].q;
                    }
                    bo.seeds_per_item = spi;
                    bo.item_rows = rows;
                    std::vector<gsi_result *> res;
                    std::vector<gsi_status> sts;
                    auto t0 = std::chrono::steady_clock::now();
                    gsi_status rc = batch_execute(g, plans, bo, res, sts);
                    if (bo.stream) cudaStreamSynchronize((cudaStream_t)bo.stream);
                    auto t1 = std::chrono::steady_clock::now();
                    for (gsi_result *r : res) delete r;
                    if (rc != GSI_OK) return rc;
                    t_best = std::min(t_best, std::chrono::duration<double, std::milli>(t1 - t0).count());
                }
                if (t_best < best) {
                    best = t_best;
                    arg_spi = spi;
                    arg_rows = rows;
                }
            }
        }
        if (best_seeds_per_item) *best_seeds_per_item = arg_spi;
        if (best_item_rows) *best_item_rows = arg_rows;
        if (best_ms) *best_ms = best;
        return GSI_OK;
    } catch (const std::bad_alloc &) {
        set_error("gsi_batch_autotune: host allocation failed");
        return GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_batch_autotune: unexpected host exception");
        return GSI_ECUDA;
    }
}

extern "C" gsi_status gsi_batch_autotune_full(gsi_graph *g, const gsi_query_desc *qs, int32_t nq,
                                              const gsi_batch_opts *opts, gsi_batch_opts *best, double *best_ms,
                                              int32_t *trials) {
    if (!g || nq < 1 || !qs || !best) {
        set_error("gsi_batch_autotune_full: need a graph, at least one query and an output");
        return GSI_EINVAL;
    }
    try {
        gsi_batch_opts bo;
        std::memset(&bo, 0, sizeof bo);
        if (opts) bo = *opts;
        bo.stats = nullptr;
        std::vector<BatchPlan> proto((size_t)nq);
        for (int32_t i = 0; i < nq; ++i)
            proto[i].status = validate_query(qs[i].vlab, qs[i].k, qs[i].src, qs[i].dst, qs[i].elab, qs[i].qm,
                                             &proto[i].q);
        int32_t runs = 0;
        // best of two runs of the calibration batch with these knobs
        auto time_of = [&](const gsi_batch_opts &o, double *ms) -> gsi_status {
            double t_best = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                std::vector<BatchPlan> plans((size_t)nq);
                for (int32_t i = 0; i < nq; ++i) {
                    plans[i].status = proto[i].status;
                    plans[i].q = proto[i].q;
                }
                std::vector<gsi_result *> res;
                std::vector<gsi_status> sts;
                auto t0 = std::chrono::steady_clock::now();
                gsi_status rc = batch_execute(g, plans, o, res, sts);
                if (o.stream) cudaStreamSynchronize((cudaStream_t)o.stream);
                auto t1 = std::chrono::steady_clock::now();
                for (gsi_result *r : res) delete r;
                ++runs;
                if (rc != GSI_OK) return rc;
                t_best = std::min(t_best, std::chrono::duration<double, std::milli>(t1 - t0).count());
            }
            *ms = t_best;
            return GSI_OK;
        };
        // coordinate descent from the defaults, one knob at a time
        gsi_batch_opts cur = bo;
        cur.seeds_per_item = 32;
        cur.item_rows = 1024;
        cur.isect = GSI_ISECT_BSEARCH;
        cur.rows_per_thread = 2;
        cur.block_threads = 256;
        double cur_ms = 0;
        GSI_TRY(time_of(cur, &cur_ms));
        auto try_knob = [&](auto set, const std::vector<int32_t> &values) -> gsi_status {
            for (int32_t v : values) {
                gsi_batch_opts cand = cur;
                set(cand, v);
                if (std::memcmp(&cand, &cur, sizeof cand) == 0) continue;
                double ms = 0;
                GSI_TRY(time_of(cand, &ms));
                if (ms < cur_ms) {
                    cur = cand;
                    cur_ms = ms;
                }
            }
            return GSI_OK;
        };
        GSI_TRY(try_knob([](gsi_batch_opts &o, int32_t v) { o.seeds_per_item = v; }, {32, 64, 128}));
        GSI_TRY(try_knob([](gsi_batch_opts &o, int32_t v) { o.item_rows = v; }, {512, 1024, 2048}));
        GSI_TRY(try_knob([](gsi_batch_opts &o, int32_t v) { o.isect = v; },
                         {GSI_ISECT_BSEARCH, GSI_ISECT_MERGE, GSI_ISECT_BITMAP}));
        GSI_TRY(try_knob(
            [](gsi_batch_opts &o, int32_t v) {
                o.block_threads = v / 10;
                o.rows_per_thread = v % 10;
            },
            {2562, 2561, 1282, 1281}));
        *best = cur;
        best->stats = opts ? opts->stats : nullptr;
        if (best_ms) *best_ms = cur_ms;
        if (trials) *trials = runs;
        return GSI_OK;
    } catch (const std::bad_alloc &) {
        set_error("gsi_batch_autotune_full: host allocation failed");
        return GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_batch_autotune_full: unexpected host exception");
        return GSI_ECUDA;
    }
}

// ------------------------------------------------------------------ server
// Admission by intermediate-table memory.  Every request carries an estimate
// of its first intermediate table: the fewest directed data edges that match
// one of its query edges by (label of one end, label of the other, edge
// label), times two int32 columns.  That is Alg. 4's preallocation bound of
// a first join step along that edge before filtering, and the planner
// usually starts where matches are scarce.  A batch reserves the sum of its
// requests' estimates times ADMIT_GROWTH (later steps' tables), each at least
// ADMIT_MIN_REQUEST (room for its result rows), and in all at least
// ADMIT_MIN_BYTES (a work area that fills every SM), out of the server's
// memory budget, allocates its work area at that size from the stream-
// ordered pool, and returns the reservation when its results are out.  A
// slot takes pending requests in arrival order while their reservation fits
// what the other slots leave free; when nothing fits it waits for a batch to
// finish.  A request too large for the budget on its own runs alone.
namespace {
constexpr uint64_t ADMIT_GROWTH = 16;
constexpr uint64_t ADMIT_MIN_BYTES = 4ull << 30;
constexpr uint64_t ADMIT_MIN_REQUEST = 1ull << 20;    // a request's share of a batch's result area, at least
constexpr size_t ADMIT_MAX_BATCH = 2048;              // requests per batch when max_batch is 0

// Directed edge counts per (label rank of v, label rank of w, edge label) of
// the CSR: one thread per vertex of the label-grouped order, one atomic per
// run of equal neighbour labels (lists are sorted by neighbour label).
__global__ void k_pair_counts(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cl,
                              const int32_t *__restrict__ gperm, int64_t np, const int64_t *__restrict__ goff,
                              int LV, int L, unsigned long long *tab) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = gperm[p];
        if (v < 0) continue;
        int lo = 0, hi = LV - 1;                    // largest r with goff[r] <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (goff[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        for (int l = 0; l < L; ++l) {
            const uint64_t seg = (uint64_t)v * (uint64_t)L + (uint64_t)l;
            uint32_t q = off[seg];
            const uint32_t e = off[seg + 1];
            while (q < e) {
                const uint16_t r2 = cl[q];
                uint32_t q2 = q + 1;
                while (q2 < e && cl[q2] == r2) ++q2;
                atomicAdd(tab + ((uint64_t)lo * (uint64_t)LV + r2) * (uint64_t)L + (uint64_t)l,
                          (unsigned long long)(q2 - q));
                q = q2;
            }
        }
    }
}
}  // namespace

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
        uint64_t est = 0;                 // estimated first intermediate table (bytes)
    };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::map<uint64_t, std::shared_ptr<Req>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    uint64_t reserved = 0;                // budget held by running batches
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<uint64_t> pair;           // directed edge counts [LV][LV][L]; empty: no estimates
};

namespace {
uint64_t estimate_bytes(const gsi_server *s, const QueryGraph &q) {
    const gsi_graph *g = s->g;
    if (s->pair.empty() || q.qm == 0) return (uint64_t)q.k * 4;     // a single vertex: its candidates
    uint64_t best = UINT64_MAX;
    for (int e = 0; e < q.qm; ++e) {
        const int32_t ra = g->label_rank(q.vl[q.src[e]]), rb = g->label_rank(q.vl[q.dst[e]]);
        const int32_t l = q.lab[e];
        uint64_t c = 0;
        if (ra >= 0 && rb >= 0 && l >= 0 && l < g->L)
            c = s->pair[((uint64_t)ra * (uint64_t)g->LV + (uint64_t)rb) * (uint64_t)g->L + (uint64_t)l];
        best = std::min(best, c);
    }
    return best * 8;
}

// A request's part of a batch reservation: its estimate grown for the later
// steps, at least ADMIT_MIN_REQUEST (its rows in the result area).
uint64_t request_need(uint64_t est) {
    const uint64_t grown = est > UINT64_MAX / ADMIT_GROWTH ? UINT64_MAX : est * ADMIT_GROWTH;
    return std::max(grown, ADMIT_MIN_REQUEST);
}
// What a batch whose requests need `need_sum` in total reserves.
uint64_t reservation(uint64_t need_sum, uint64_t budget) { return std::min(budget, std::max(need_sum, ADMIT_MIN_BYTES)); }
}  // namespace

// The work of one slot's take: requests one by one on the plain path, or as
// one batch in a work area of `reserve` bytes (allocated here, stream-ordered,
// and released once the results are gathered out of it).
template <class Publish>
static void serve_batch(gsi_server *s, cudaStream_t st, uint64_t reserve, size_t max_batch, size_t min_batch,
                        std::vector<std::shared_ptr<gsi_server::Req>> &batch, std::vector<gsi_result *> &res,
                        std::vector<gsi_status> &sts, Publish &publish) {
    if (max_batch == 1 || batch.size() < min_batch) {
        // too few requests to fill the GPU with (query, seed range) items:
        // one query at a time on the plain path, every step on all SMs
        for (size_t i = 0; i < batch.size(); ++i) {
            gsi_query_opts o;
            std::memset(&o, 0, sizeof o);
            o.stream = st;
            o.row_cap = s->opts.row_cap;
            o.count_only = s->opts.count_only;
            o.mem_budget = reserve;
            sts[i] = run_query(s->g, batch[i]->q, o, &res[i]);
            publish(i, i + 1);
        }
        return;
    }
    BatchWorkspace ws;
    ws.result_bytes = (reserve / 5) / 256 * 256;
    ws.arena_bytes = (reserve - ws.result_bytes) / 256 * 256;
    if (cudaMallocAsync((void **)&ws.arena, ws.arena_bytes, st) != cudaSuccess ||
        cudaMallocAsync((void **)&ws.result, ws.result_bytes, st) != cudaSuccess) {
        (void)cudaGetLastError();
        if (ws.arena) cudaFreeAsync(ws.arena, st);
        ws = BatchWorkspace();             // the batch reserves its own memory
    }
    std::vector<BatchPlan> plans(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) plans[i].q = batch[i]->q;
    gsi_batch_opts bo;
    std::memset(&bo, 0, sizeof bo);
    bo.stream = st;
    bo.row_cap = s->opts.row_cap;
    bo.mem_budget = reserve;
    bo.count_only = s->opts.count_only;
    bo.seeds_per_item = s->opts.seeds_per_item;
    bo.item_rows = s->opts.item_rows;
    bo.isect = s->opts.isect;
    bo.rows_per_thread = s->opts.rows_per_thread;
    bo.block_threads = s->opts.block_threads;
    gsi_status rc = batch_execute(s->g, plans, bo, res, sts, ws.arena ? &ws : nullptr);
    if (ws.arena) cudaFreeAsync(ws.arena, st);      // results were gathered into their own buffers
    if (ws.result) cudaFreeAsync(ws.result, st);
    if (rc != GSI_OK)
        for (size_t i = 0; i < batch.size(); ++i)
            if (sts[i] == GSI_OK && !res[i]) sts[i] = rc;
    publish(0, batch.size());
}

// One slot: a worker thread with its own stream.  It takes pending requests
// in arrival order (up to max_batch) while the batch's reservation fits the
// memory the other slots leave free, so requests that arrived while other
// batches were on the GPU are admitted as soon as a slot and memory free up;
// batches of different slots overlap on the device.  With max_batch == 1, or
// fewer than min_batch requests taken, a slot runs one query at a time on the
// plain path.
static void server_worker(gsi_server *s, int idx) {
    cudaSetDevice(s->g->device);
    cudaStream_t st = s->streams[idx];
    const uint64_t budget = s->opts.mem_budget;
    const size_t max_batch = s->opts.max_batch > 0 ? (size_t)s->opts.max_batch : ADMIT_MAX_BATCH;
    const size_t min_batch = s->opts.min_batch > 0 ? (size_t)s->opts.min_batch : 16;
    for (;;) {
        std::vector<std::shared_ptr<gsi_server::Req>> batch;
        bool cancelled = false;
        uint64_t reserve = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // work to do and memory for at least the first request
            auto admissible = [&] {
                while (!s->queue.empty() && s->queue.front()->cancelled) {
                    s->queue.front()->status = GSI_ECANCELLED;
                    s->queue.pop_front();
                    cancelled = true;
                }
                if (s->queue.empty()) return false;
                const uint64_t need = reservation(request_need(s->queue.front()->est), budget);
                return s->reserved == 0 || s->reserved + need <= budget;
            };
            s->cv_work.wait(lk, [&] { return s->stop || admissible(); });
            if (s->stop && s->queue.empty()) return;
            uint64_t need_sum = 0;
            while (!s->queue.empty() && batch.size() < max_batch) {
                auto r = s->queue.front();
                if (r->cancelled) {
                    r->status = GSI_ECANCELLED;
                    s->queue.pop_front();
                    cancelled = true;
                    continue;
                }
                const uint64_t need = reservation(need_sum + request_need(r->est), budget);
                if (!batch.empty() && s->reserved + need > budget) break;     // arrival order: wait for memory
                need_sum += request_need(r->est);
                batch.push_back(r);
                s->queue.pop_front();
            }
            if (!batch.empty()) {
                reserve = reservation(need_sum, budget);
                if (s->reserved + reserve > budget)      // a request larger than what is free runs alone
                    reserve = budget > s->reserved ? budget - s->reserved : reserve;
                s->reserved += reserve;
            }
        }
        if (cancelled) s->cv_done.notify_all();     // their pollers need not wait for this batch
        if (batch.empty()) continue;
        std::vector<gsi_result *> res(batch.size(), nullptr);
        std::vector<gsi_status> sts(batch.size(), GSI_OK);
        size_t published = 0;                        // requests [0, published) have their outcome
        // hand results [lo, hi) to their requests
        auto publish = [&](size_t lo, size_t hi) {
            auto now = std::chrono::steady_clock::now();
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (size_t i = lo; i < hi; ++i) {
                    if (res[i]) {                  // slot streams are the server's: release elsewhere
                        res[i]->own_stream = false;
                        if (res[i]->arena) res[i]->arena->own_stream = false;
                    }
                    batch[i]->res = res[i];
                    batch[i]->status = sts[i];
                    batch[i]->latency_ms = std::chrono::duration<double, std::milli>(now - batch[i]->t_submit).count();
                }
                published = hi;
            }
            s->cv_done.notify_all();
        };
        try {
            serve_batch(s, st, reserve, max_batch, min_batch, batch, res, sts, publish);
        } catch (...) {
            // a host exception (allocation) must not leave the thread: the
            // requests not yet answered fail, and results made for them are freed
            gsi_status fail = GSI_ECUDA;
            try {
                throw;
            } catch (const std::bad_alloc &) {
                fail = GSI_ENOMEM;
            } catch (...) {
            }
            res.resize(batch.size(), nullptr);
            sts.resize(batch.size(), fail);
            for (size_t i = published; i < batch.size(); ++i) {
                if (res[i]) gsi_result_destroy(res[i]);
                res[i] = nullptr;
                sts[i] = fail;
            }
            publish(published, batch.size());
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->reserved -= reserve;
        }
        s->cv_work.notify_all();                     // memory freed: waiting slots may admit
    }
}

// Stop the slots after the queue drains, then release every resource the
// server holds (also a partly created one).
static void server_teardown(gsi_server *s) {
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

// The directed edge counts per (label, label, edge label) behind the
// admission estimates, when the table stays small.
static gsi_status pair_counts(gsi_server *s) {
    gsi_graph *g = s->g;
    const uint64_t cells = (uint64_t)g->LV * (uint64_t)g->LV * (uint64_t)g->L;
    if (g->m == 0 || g->np == 0 || cells > (1ull << 24)) return GSI_OK;      // no estimates: minimal reservations
    unsigned long long *tab = nullptr;
    int64_t *goff = nullptr;
    cudaStream_t st = s->streams[0];
    GSI_CUDA_TRY(cudaMallocAsync(&tab, cells * 8, st));
    gsi_status rc = GSI_OK;
    if (cudaMallocAsync(&goff, sizeof(int64_t) * g->goff.size(), st) != cudaSuccess ||
        cudaMemsetAsync(tab, 0, cells * 8, st) != cudaSuccess ||
        cudaMemcpyAsync(goff, g->goff.data(), sizeof(int64_t) * g->goff.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
        set_error("gsi_server_create: pair-count table setup failed");
        rc = GSI_ECUDA;
    }
    if (rc == GSI_OK) {
        const int blocks = (int)std::min<int64_t>((g->np + 255) / 256, 4096);
        k_pair_counts<<<blocks, 256, 0, st>>>(g->off, g->cl, g->gperm, g->np, goff, g->LV, g->L, tab);
        s->pair.resize(cells);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(s->pair.data(), tab, cells * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("gsi_server_create: pair-count kernel failed");
            s->pair.clear();
            rc = GSI_ECUDA;
        }
    }
    cudaFreeAsync(tab, st);
    if (goff) cudaFreeAsync(goff, st);
    cudaStreamSynchronize(st);
    return rc;
}

static gsi_status server_start(gsi_server *s) {
    if (s->opts.n_streams < 1) s->opts.n_streams = 2;
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
    GSI_TRY(pair_counts(s));
    for (int i = 0; i < s->opts.n_streams; ++i) s->workers.emplace_back(server_worker, s, i);
    return GSI_OK;
}

extern "C" gsi_status gsi_server_create(gsi_graph *g, const gsi_server_opts *opts, gsi_server **out) {
    if (!g || !out) {
        set_error("gsi_server_create: null argument");
        return GSI_EINVAL;
    }
    *out = nullptr;
    GSI_TRY(prepare_device(g->device));
    gsi_server *s = nullptr;
    gsi_status rc = GSI_ECUDA;
    try {
        s = new gsi_server();
        s->g = g;
        std::memset(&s->opts, 0, sizeof s->opts);
        if (opts) s->opts = *opts;
        rc = server_start(s);
    } catch (const std::bad_alloc &) {
        set_error("gsi_server_create: host allocation failed");
        rc = GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_server_create: could not start the worker threads");
        rc = GSI_ECUDA;
    }
    if (rc != GSI_OK) {
        if (s) server_teardown(s);
        return rc;
    }
    *out = s;
    return GSI_OK;
}

extern "C" gsi_status gsi_server_submit(gsi_server *s, const gsi_query_desc *q, uint64_t *ticket) {
    if (!s || !q || !ticket) {
        set_error("gsi_server_submit: null argument");
        return GSI_EINVAL;
    }
    try {
        auto r = std::make_shared<gsi_server::Req>();
        GSI_TRY(validate_query(q->vlab, q->k, q->src, q->dst, q->elab, q->qm, &r->q));
        r->est = estimate_bytes(s, r->q);
        r->t_submit = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->all[s->next_ticket] = r;              // may throw: the ticket is taken only after
            s->queue.push_back(r);
            r->ticket = s->next_ticket++;
        }
        s->cv_work.notify_one();
        *ticket = r->ticket;
        return GSI_OK;
    } catch (const std::bad_alloc &) {
        set_error("gsi_server_submit: host allocation failed");
        return GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_server_submit: unexpected host exception");
        return GSI_ECUDA;
    }
}

extern "C" gsi_status gsi_server_estimate(gsi_server *s, const gsi_query_desc *q, uint64_t *bytes) {
    if (!s || !q || !bytes) {
        set_error("gsi_server_estimate: null argument");
        return GSI_EINVAL;
    }
    try {
        QueryGraph qg;
        GSI_TRY(validate_query(q->vlab, q->k, q->src, q->dst, q->elab, q->qm, &qg));
        *bytes = estimate_bytes(s, qg);
        return GSI_OK;
    } catch (...) {
        set_error("gsi_server_estimate: host allocation failed");
        return GSI_ENOMEM;
    }
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
    if (s) server_teardown(s);
}

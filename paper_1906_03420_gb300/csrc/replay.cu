// Prepared batches: a batch planned once and replayed from a captured CUDA
// graph.
//
// gsi_batch_prepare runs the batched filter once, plans every query (Alg. 2
// order, join steps), reserves the control block and the work area, and
// captures the device work of one pass into a CUDA graph: the filter (bitmaps
// zeroed, Sec. III-A test for every query vertex) and the batch kernel (query
// records reset from a device template, spill queue cleared, k_batch).  Each
// gsi_batch_replay reserves a fresh result arena, writes the launch's control
// words, launches the graph, reads the outcome back and hands out results;
// queries that did not fit the batch run again on the plain path.  Every
// replay recomputes the filter and the whole join on the device; what it
// reuses is host work whose outcome is fixed by the inputs (validation,
// signatures, the order of Alg. 2 from the candidate counts, the step
// configurations).
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "runtime.h"

using namespace gsi;

struct gsi_batch {
    gsi_graph *g = nullptr;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    gsi_batch_opts opts;
    uint64_t budget = 0;
    std::vector<BatchPlan> plans;
    BatchInputs in;
    BatchLaunch L;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    ~gsi_batch();
};

gsi_batch::~gsi_batch() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (g && cur != g->device) cudaSetDevice(g->device);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (st) {
        batch_release(L, st);
        batch_inputs_free(in, st);
        cudaStreamSynchronize(st);
        if (own_stream) cudaStreamDestroy(st);
    }
    if (g && cur >= 0 && cur != g->device) cudaSetDevice(cur);
}

extern "C" gsi_status gsi_batch_prepare(gsi_graph *g, const gsi_query_desc *qs, int32_t nq,
                                        const gsi_batch_opts *opts, gsi_batch **out, int32_t *statuses) {
    if (!g || !out || nq < 0 || (nq > 0 && !qs)) {
        set_error("gsi_batch_prepare: null argument");
        return GSI_EINVAL;
    }
    *out = nullptr;
    try {
        GSI_TRY(prepare_device(g->device));
        std::unique_ptr<gsi_batch> b(new gsi_batch());
        b->g = g;
        std::memset(&b->opts, 0, sizeof b->opts);
        if (opts) b->opts = *opts;
        const bool counters = opts && opts->stats;   // count algorithmic bytes in the kernels
        b->opts.stats = nullptr;                 // replays take their own
        if (b->opts.stream) {
            b->st = (cudaStream_t)b->opts.stream;
        } else {                                 // the legacy stream cannot be captured
            GSI_CUDA_TRY(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
            b->own_stream = true;
        }
        b->budget = batch_budget(b->opts);
        b->plans.resize((size_t)nq);
        for (int32_t i = 0; i < nq; ++i) {
            b->plans[i].status = validate_query(qs[i].vlab, qs[i].k, qs[i].src, qs[i].dst, qs[i].elab, qs[i].qm,
                                                &b->plans[i].q);
            if (statuses) statuses[i] = b->plans[i].status;
        }
        GSI_TRY(batch_plan_all(g, b->plans, nullptr, b->st, b->in));
        GSI_TRY(batch_setup(b->L, g, b->plans, b->opts, b->budget, b->st, nullptr, counters, true));
        for (cudaEvent_t &e : b->ev) GSI_CUDA_TRY(cudaEventCreate(&e));
        GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
        // one pass of device work, captured
        GSI_CUDA_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        gsi_status rc = GSI_OK;
        if (cudaEventRecordWithFlags(b->ev[0], b->st, cudaEventRecordExternal) != cudaSuccess) rc = GSI_ECUDA;
        if (rc == GSI_OK) rc = filter_enqueue(g, b->in.fp, b->in.bitmaps, b->in.counts, b->st);
        if (rc == GSI_OK && cudaEventRecordWithFlags(b->ev[1], b->st, cudaEventRecordExternal) != cudaSuccess)
            rc = GSI_ECUDA;
        if (rc == GSI_OK) rc = batch_enqueue_kernel(b->L, b->st);
        if (rc == GSI_OK && cudaEventRecordWithFlags(b->ev[2], b->st, cudaEventRecordExternal) != cudaSuccess)
            rc = GSI_ECUDA;
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(b->st, &graph);
        b->graph = graph;
        if (rc != GSI_OK || ce != cudaSuccess || !graph) {
            (void)cudaGetLastError();
            set_error("gsi_batch_prepare: capturing the batch into a CUDA graph failed");
            return rc != GSI_OK ? rc : GSI_ECUDA;
        }
        GSI_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
        *out = b.release();
        return GSI_OK;
    } catch (const std::bad_alloc &) {
        set_error("gsi_batch_prepare: host allocation failed");
        return GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_batch_prepare: unexpected host exception");
        return GSI_ECUDA;
    }
}

extern "C" gsi_status gsi_batch_replay(gsi_batch *b, gsi_result **outs, int32_t *statuses, gsi_stats *stats) {
    if (!b || (!b->plans.empty() && !outs)) {
        set_error("gsi_batch_replay: null argument");
        return GSI_EINVAL;
    }
    try {
        gsi_graph *g = b->g;
        GSI_TRY(prepare_device(g->device));
        cudaStream_t st = b->st;
        int32_t *result = nullptr;
        std::shared_ptr<ResultArena> arena;
        if (!b->L.all_plain && b->L.result_bytes) {
            if (cudaMallocAsync(&result, b->L.result_bytes, st) != cudaSuccess) {
                (void)cudaGetLastError();
                set_error("gsi_batch_replay: could not reserve the result arena");
                return GSI_ENOMEM;
            }
            arena = std::make_shared<ResultArena>();     // the last result to go releases it
            arena->ptr = result;
            arena->device = g->device;
            arena->stream = st;
            arena->own_stream = !b->own_stream;           // a private stream dies with the batch
        }
        GSI_TRY(batch_enqueue_ctl(b->L, result, b->L.result_bytes, st));
        GSI_CUDA_TRY(cudaGraphLaunch(b->exec, st));
        gsi_status rc = batch_collect(b->L, g, b->plans, result, arena, st, stats, nullptr);
        if (rc != GSI_OK) return rc;
        if (stats) {
            float fms = 0, jms = 0;
            cudaEventElapsedTime(&fms, b->ev[0], b->ev[1]);
            cudaEventElapsedTime(&jms, b->ev[1], b->ev[2]);
            stats->filter_ms += fms;
            stats->join_ms += jms;
            stats->batch_ms += jms;
            stats->filter_launches += b->in.fp.ngroups ? 1 : 0;
            stats->join_launches += b->L.nitems ? 1 : 0;
            stats->kernels += (b->in.fp.ngroups ? 1 : 0) + (b->L.nitems ? 1 : 0);
            stats->filter_bytes += filter_alg_bytes(g, b->in.labels);
        }
        gsi_batch_opts bo = b->opts;
        bo.stats = stats;
        std::vector<gsi_result *> res;
        std::vector<gsi_status> sts;
        rc = batch_finish(g, b->plans, bo, b->budget, st, res, sts);
        for (size_t i = 0; i < res.size(); ++i) {
            if (res[i] && b->own_stream) {                // released on the library stream
                res[i]->own_stream = false;
                if (res[i]->arena) res[i]->arena->own_stream = false;
            }
            outs[i] = res[i];
            if (statuses) statuses[i] = sts[i];
        }
        return rc;
    } catch (const std::bad_alloc &) {
        set_error("gsi_batch_replay: host allocation failed");
        return GSI_ENOMEM;
    } catch (...) {
        set_error("gsi_batch_replay: unexpected host exception");
        return GSI_ECUDA;
    }
}

extern "C" void gsi_batch_destroy(gsi_batch *b) { delete b; }

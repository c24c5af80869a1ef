// extern "C" entry points of include/gsi.h.
#include <cstring>
#include <memory>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "runtime.h"

using namespace gsi;

// Result memory is released stream-ordered on a library stream: cudaFree
// would wait for every kernel on the device, stalling concurrent queries.
// The producing stream has always completed before a result is handed out.
static cudaStream_t release_stream(int dev) {
    static std::mutex mu;
    static cudaStream_t streams[64];
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

gsi_result::~gsi_result() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    cudaStream_t rs = own_stream ? stream : release_stream(device);
    for (auto &c : chunks) {
        if (c.owned) cudaFreeAsync(c.rows, rs);
        if (c.held) gsi::release_region(device, c.held);
    }
    arena.reset();
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
}

gsi::ResultArena::~ResultArena() {
    if (!ptr) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    cudaFreeAsync(ptr, own_stream ? stream : release_stream(device));
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
}

namespace gsi {
gsi_status join_step_args(const char *who, gsi_graph *g, const int32_t *M, uint64_t R, int32_t t,
                          const uint32_t *cand, int32_t ulabel, const int32_t *col, const int32_t *lab, int32_t d,
                          int32_t *out, uint64_t out_cap, uint64_t *count, JoinStep *s, bool *empty) {
    if (!g || !count || !col || !lab || (R > 0 && (!M || !cand)) || (out_cap > 0 && !out)) {
        set_error(std::string(who) + ": null argument");
        return GSI_EINVAL;
    }
    if (t < 1 || t >= GSI_MAX_QUERY_VERTICES || d < 1 || d > t) {
        set_error(std::string(who) + ": need 1 <= d <= t < 32");
        return GSI_EINVAL;
    }
    s->t = t;
    s->d = d;
    s->ulab = g->label_rank(ulabel);
    bool none = s->ulab < 0;
    for (int j = 0; j < d; ++j) {
        if (col[j] < 0 || col[j] >= t || lab[j] < 0) {
            set_error(std::string(who) + ": column out of range or negative label");
            return GSI_EINVAL;
        }
        s->col[j] = col[j];
        s->lab[j] = lab[j];
        none |= lab[j] >= g->L;
    }
    for (int c = 0; c <= t; ++c) s->perm[c] = c;
    *count = 0;
    *empty = R == 0 || none;
    return GSI_OK;
}
}  // namespace gsi

extern "C" {

const char *gsi_version(void) { return "gsi-gb300 0.1 (sm_103a)"; }

gsi_status gsi_graph_create(const int32_t *vlab, int32_t n, const int32_t *src, const int32_t *dst,
                            const int32_t *elab, int64_t m, const gsi_graph_opts *opts, gsi_graph **out) {
    GSI_API_BEGIN
    if (!out) {
        set_error("gsi_graph_create: null out");
        return GSI_EINVAL;
    }
    *out = nullptr;
    int dev = opts ? opts->device : 0;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
    GSI_TRY(prepare_device(dev));
    std::unique_ptr<gsi_graph> g(new gsi_graph());
    g->device = dev;
    gsi_status rc = build_graph(g.get(), vlab, n, src, dst, elab, m, st);
    if (rc != GSI_OK) {
        if (g->off) cudaFree(g->off);
        if (g->ci) cudaFree(g->ci);
        if (g->cl) cudaFree(g->cl);
        if (g->sig) cudaFree(g->sig);
        if (g->gperm) cudaFree(g->gperm);
        if (g->gsig) cudaFree(g->gsig);
        return rc;
    }
    *out = g.release();
    return GSI_OK;
    GSI_API_END
}

void gsi_graph_destroy(gsi_graph *g) {
    if (!g) return;
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->off);
    cudaFree(g->ci);
    cudaFree(g->cl);
    cudaFree(g->sig);
    cudaFree(g->gperm);
    cudaFree(g->gsig);
    if (cur >= 0) cudaSetDevice(cur);
    delete g;
}

gsi_status gsi_graph_get_info(const gsi_graph *g, gsi_graph_info *info) {
    if (!g || !info) {
        set_error("gsi_graph_get_info: null argument");
        return GSI_EINVAL;
    }
    info->n = g->n;
    info->n_elabels = g->L;
    info->m = g->m;
    info->device_bytes = g->device_bytes;
    info->build_ms = g->build_ms;
    info->off = g->off;
    info->ci = g->ci;
    info->cl = g->cl;
    info->sig = g->sig;
    info->n_vlabels = g->LV;
    return GSI_OK;
}

gsi_status gsi_graph_export(const gsi_graph *g, uint32_t *off, int32_t *ci, uint16_t *cl, uint32_t *sig) {
    if (!g) {
        set_error("gsi_graph_export: null graph");
        return GSI_EINVAL;
    }
    GSI_CUDA_TRY(cudaSetDevice(g->device));
    const uint64_t nseg = (uint64_t)g->n * (uint64_t)g->L;
    if (off) GSI_CUDA_TRY(cudaMemcpy(off, g->off, 4 * (nseg + 1), cudaMemcpyDefault));
    if (ci && g->m > 0) GSI_CUDA_TRY(cudaMemcpy(ci, g->ci, 8 * (uint64_t)g->m, cudaMemcpyDefault));
    if (cl && g->m > 0) GSI_CUDA_TRY(cudaMemcpy(cl, g->cl, 4 * (uint64_t)g->m, cudaMemcpyDefault));
    if (sig) GSI_CUDA_TRY(cudaMemcpy(sig, g->sig, 4ull * GSI_SIG_WORDS * (uint64_t)g->n, cudaMemcpyDefault));
    return GSI_OK;
}

gsi_status gsi_graph_label_freq(const gsi_graph *g, uint64_t *freq, int32_t max_labels) {
    if (!g || !freq || max_labels < 0) {
        set_error("gsi_graph_label_freq: bad argument");
        return GSI_EINVAL;
    }
    for (int32_t l = 0; l < max_labels; ++l) freq[l] = l < g->L ? g->freq[l] : 0;
    return GSI_OK;
}

gsi_status gsi_query_run(gsi_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                         const int32_t *qelab, int32_t qm, const gsi_query_opts *opts, gsi_result **out) {
    GSI_API_BEGIN
    if (!g || !out) {
        set_error("gsi_query_run: null graph or out");
        return GSI_EINVAL;
    }
    *out = nullptr;
    QueryGraph q;
    GSI_TRY(validate_query(qvlab, k, qsrc, qdst, qelab, qm, &q));
    gsi_query_opts o;
    std::memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.semantics != GSI_ISOMORPHISM && o.semantics != GSI_HOMOMORPHISM) {
        set_error("gsi_query_run: unsupported semantics");
        return GSI_EINVAL;
    }
    return run_query(g, q, o, out);
    GSI_API_END
}

gsi_status gsi_result_count(const gsi_result *r, uint64_t *count) {
    if (!r || !count) {
        set_error("gsi_result_count: null argument");
        return GSI_EINVAL;
    }
    *count = r->count;
    return GSI_OK;
}

gsi_status gsi_result_columns(const gsi_result *r, int32_t *k) {
    if (!r || !k) {
        set_error("gsi_result_columns: null argument");
        return GSI_EINVAL;
    }
    *k = r->k;
    return GSI_OK;
}

gsi_status gsi_result_copy(const gsi_result *r, int32_t *dst, uint64_t max_rows, uint64_t *rows) {
    if (!r || (!dst && max_rows > 0)) {
        set_error("gsi_result_copy: null argument");
        return GSI_EINVAL;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != r->device) cudaSetDevice(r->device);
    uint64_t done = 0;
    for (const auto &c : r->chunks) {
        if (done >= max_rows) break;
        uint64_t take = std::min<uint64_t>(c.nrows, max_rows - done);
        cudaError_t e = cudaMemcpy(dst + done * (uint64_t)r->k, c.rows, take * (uint64_t)r->k * 4, cudaMemcpyDefault);
        if (e != cudaSuccess) {
            set_error(std::string("gsi_result_copy: ") + cudaGetErrorString(e));
            if (cur >= 0 && cur != r->device) cudaSetDevice(cur);
            return GSI_ECUDA;
        }
        done += take;
    }
    if (cur >= 0 && cur != r->device) cudaSetDevice(cur);
    if (rows) *rows = done;
    return r->materialised < r->count ? GSI_ECAPPED : GSI_OK;
}

gsi_status gsi_result_copy_async(const gsi_result *r, int32_t *dst, uint64_t max_rows, uint64_t *rows,
                                 void *stream) {
    if (!r || (!dst && max_rows > 0)) {
        set_error("gsi_result_copy_async: null argument");
        return GSI_EINVAL;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != r->device) cudaSetDevice(r->device);
    uint64_t done = 0;
    for (const auto &c : r->chunks) {
        if (done >= max_rows) break;
        uint64_t take = std::min<uint64_t>(c.nrows, max_rows - done);
        cudaError_t e = cudaMemcpyAsync(dst + done * (uint64_t)r->k, c.rows, take * (uint64_t)r->k * 4,
                                        cudaMemcpyDefault, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            set_error(std::string("gsi_result_copy_async: ") + cudaGetErrorString(e));
            if (cur >= 0 && cur != r->device) cudaSetDevice(cur);
            return GSI_ECUDA;
        }
        done += take;
    }
    if (cur >= 0 && cur != r->device) cudaSetDevice(cur);
    if (rows) *rows = done;
    return r->materialised < r->count ? GSI_ECAPPED : GSI_OK;
}

void gsi_result_destroy(gsi_result *r) { delete r; }

gsi_status gsi_query_signatures(const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                                const int32_t *qelab, int32_t qm, uint32_t *sig) {
    GSI_API_BEGIN
    if (!sig) {
        set_error("gsi_query_signatures: null output");
        return GSI_EINVAL;
    }
    QueryGraph q;
    // signatures do not need a connected query
    if (k < 1 || k > GSI_MAX_QUERY_VERTICES || !qvlab || qm < 0) {
        set_error("gsi_query_signatures: bad query");
        return GSI_EINVAL;
    }
    for (int e = 0; e < qm; ++e)
        if (qsrc[e] < 0 || qsrc[e] >= k || qdst[e] < 0 || qdst[e] >= k || qsrc[e] == qdst[e]) {
            set_error("gsi_query_signatures: bad edge");
            return GSI_EINVAL;
        }
    QuerySig qs;
    query_signatures(qvlab, k, qsrc, qdst, qelab, qm, &qs);
    for (int u = 0; u < k; ++u) std::memcpy(sig + u * GSI_SIG_WORDS, qs.sig[u], sizeof(uint32_t) * GSI_SIG_WORDS);
    (void)q;
    return GSI_OK;
    GSI_API_END
}

gsi_status gsi_filter(gsi_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                      const int32_t *qelab, int32_t qm, uint32_t *bitmaps, uint64_t *counts, void *stream) {
    GSI_API_BEGIN
    if (!g || !bitmaps || !counts) {
        set_error("gsi_filter: null argument");
        return GSI_EINVAL;
    }
    QueryGraph q;
    GSI_TRY(validate_query(qvlab, k, qsrc, qdst, qelab, qm, &q));
    GSI_TRY(prepare_device(g->device));
    cudaStream_t st = (cudaStream_t)stream;
    QuerySig qs;
    query_signatures(qvlab, k, qsrc, qdst, qelab, qm, &qs);
    uint32_t *d_bm = nullptr;
    unsigned long long *d_cnt = nullptr;
    const uint64_t words = (uint64_t)k * (uint64_t)g->nwords;
    GSI_CUDA_TRY(cudaMallocAsync(&d_bm, words * 4 + 16, st));
    GSI_CUDA_TRY(cudaMallocAsync(&d_cnt, 8 * (size_t)k, st));
    gsi_status rc = launch_filter(g, qs, d_bm, d_cnt, st);
    if (rc == GSI_OK) {
        if (cudaMemcpyAsync(bitmaps, d_bm, words * 4, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaMemcpyAsync(counts, d_cnt, 8 * (size_t)k, cudaMemcpyDefault, st) != cudaSuccess) {
            set_error("gsi_filter: copy-out failed");
            rc = GSI_ECUDA;
        }
    }
    cudaFreeAsync(d_bm, st);
    cudaFreeAsync(d_cnt, st);
    GSI_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
    GSI_API_END
}

gsi_status gsi_join_step(gsi_graph *g, const int32_t *M, uint64_t R, int32_t t, const uint32_t *cand,
                         int32_t ulabel, const int32_t *col, const int32_t *lab, int32_t d, int32_t *out,
                         uint64_t out_cap, uint64_t *count, void *stream) {
    GSI_API_BEGIN
    JoinStep s;
    bool empty = false;
    GSI_TRY(join_step_args("gsi_join_step", g, M, R, t, cand, ulabel, col, lab, d, out, out_cap, count, &s, &empty));
    if (empty) return GSI_OK;
    GSI_TRY(prepare_device(g->device));
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *F = nullptr, *scr = nullptr;
    uint64_t h[2] = {0, 0};
    int64_t *part = nullptr;
    unsigned long long *d_cnt = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync(&F, 8 * (R + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&scr, 8 * (uint64_t)join_scan_scratch(R), st));
    GSI_CUDA_TRY(cudaMallocAsync(&d_cnt, 8, st));
    gsi_status rc = launch_join_scan(g, M, R, s, F, scr, st);
    uint64_t total = 0;
    if (rc == GSI_OK) {
        if (cudaMemcpyAsync(h, F + R, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("gsi_join_step: readback failed");
            rc = GSI_ECUDA;
        }
        total = h[0];
    }
    if (rc == GSI_OK) {
        const uint64_t ntiles = join_tiles(total);
        if (cudaMallocAsync(&part, 8 * (ntiles + 1), st) != cudaSuccess ||
            cudaMemsetAsync(d_cnt, 0, 8, st) != cudaSuccess) {
            set_error("gsi_join_step: scratch allocation failed");
            rc = GSI_ENOMEM;
        }
    }
    if (rc == GSI_OK) rc = launch_partition(F, R, total, part, st);
    if (rc == GSI_OK)
        rc = launch_join(g, M, R, s, F, total, part, cand, out, out_cap, d_cnt, out_cap == 0 ? 1 : 0, nullptr, st);
    if (rc == GSI_OK) {
        if (cudaMemcpyAsync(h, d_cnt, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("gsi_join_step: kernel or readback failed");
            rc = GSI_ECUDA;
        } else {
            *count = h[0];
        }
    }
    cudaFreeAsync(F, st);
    cudaFreeAsync(scr, st);
    if (part) cudaFreeAsync(part, st);
    cudaFreeAsync(d_cnt, st);
    cudaStreamSynchronize(st);
    return rc;
    GSI_API_END
}

gsi_status gsi_plan_order(int32_t k, const int32_t *qsrc, const int32_t *qdst, const int32_t *qelab, int32_t qm,
                          const uint64_t *cand, const uint64_t *freq, int32_t n_labels, int32_t *order_out,
                          int32_t *first_edge) {
    GSI_API_BEGIN
    if (!cand || !freq || !order_out || !first_edge || n_labels < 0) {
        set_error("gsi_plan_order: null argument");
        return GSI_EINVAL;
    }
    int32_t vl[GSI_MAX_QUERY_VERTICES] = {0};
    QueryGraph q;
    GSI_TRY(validate_query(vl, k, qsrc, qdst, qelab, qm, &q));
    plan_order(q, cand, freq, n_labels, order_out, first_edge);
    return GSI_OK;
    GSI_API_END
}

gsi_status gsi_selftest_wait_timeout(int32_t device, uint64_t spin_limit, double *elapsed_ms) {
    GSI_API_BEGIN
    GSI_TRY(prepare_device(device));
    return selftest_barrier_timeout(device, spin_limit ? spin_limit : 4096, elapsed_ms);
    GSI_API_END
}

}  // extern "C"

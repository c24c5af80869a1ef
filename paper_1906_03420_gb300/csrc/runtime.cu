// Host runtime behind the C ABI: graph objects, query validation, the Alg. 2
// planner, the memory-bounded depth-first join driver and result objects.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "runtime.h"

int32_t gsi_graph::label_rank(int32_t label) const {
    auto it = std::lower_bound(vlabels.begin(), vlabels.end(), label);
    if (it == vlabels.end() || *it != label) return -1;
    return (int32_t)(it - vlabels.begin());
}

namespace gsi {

static thread_local std::string t_last_error;
void set_error(const std::string &msg) { t_last_error = msg; }
const char *last_error() { return t_last_error.c_str(); }

// --------------------------------------------------------------- devices
static std::once_flag g_pool_once[64];

gsi_status prepare_device(int dev) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        set_error("no CUDA device available");
        return GSI_ECUDA;
    }
    if (dev < 0 || dev >= ndev) {
        set_error("device ordinal out of range");
        return GSI_EINVAL;
    }
    GSI_CUDA_TRY(cudaSetDevice(dev));
    // a failed call of an earlier request leaves a non-sticky error behind;
    // clear it so that launch checks below report only this request's errors
    (void)cudaGetLastError();
    if (dev < 64) {
        std::call_once(g_pool_once[dev], [dev]() {
            // keep freed stream-ordered blocks cached for reuse by later queries
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        });
    }
    return GSI_OK;
}

// ------------------------------------------------------- query validation
gsi_status validate_query(const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                          const int32_t *qelab, int32_t qm, QueryGraph *q) {
    if (k < 1 || k > GSI_MAX_QUERY_VERTICES) {
        set_error("query: need 1 <= k <= 32");
        return GSI_EINVAL;
    }
    if (qm < 0 || (qm > 0 && (!qsrc || !qdst || !qelab)) || !qvlab) {
        set_error("query: null arrays or negative edge count");
        return GSI_EINVAL;
    }
    q->k = k;
    for (int u = 0; u < k; ++u) {
        q->vlab[u] = qvlab[u];
        for (int w = 0; w < k; ++w) q->elab[u][w] = -1;
    }
    for (int e = 0; e < qm; ++e) {
        int a = qsrc[e], b = qdst[e];
        if (a < 0 || a >= k || b < 0 || b >= k) {
            set_error("query: vertex id out of range");
            return GSI_EINVAL;
        }
        if (a == b) {
            set_error("query: self-loop");
            return GSI_EINVAL;
        }
        if (qelab[e] < 0) {
            set_error("query: negative edge label");
            return GSI_EINVAL;
        }
        if (q->elab[a][b] >= 0) {
            set_error("query: vertex pair given twice");
            return GSI_EINVAL;
        }
        q->elab[a][b] = q->elab[b][a] = qelab[e];
    }
    // connectivity (the paper assumes a connected query, Sec. II-A)
    uint32_t seen = 1u, frontier = 1u;
    while (frontier) {
        uint32_t next = 0;
        for (int u = 0; u < k; ++u)
            if ((frontier >> u) & 1u)
                for (int w = 0; w < k; ++w)
                    if (q->elab[u][w] >= 0 && !((seen >> w) & 1u)) next |= 1u << w;
        seen |= next;
        frontier = next;
    }
    uint32_t all = k == 32 ? 0xffffffffu : ((1u << k) - 1u);
    if (seen != all) {
        set_error("query: not connected");
        return GSI_EINVAL;
    }
    q->qm = qm;
    q->src.assign(qsrc, qsrc + qm);
    q->dst.assign(qdst, qdst + qm);
    q->lab.assign(qelab, qelab + qm);
    q->vl.assign(qvlab, qvlab + k);
    return GSI_OK;
}

// --------------------------------------------------------------- planner
// Alg. 2: score(u) = |C(u)| / deg(u); start at the minimum; then repeatedly
// take the unmatched vertex of least score adjacent to the matched part, and
// after each pick multiply its neighbours' scores by freq(label of the edge).
// Alg. 4: the first edge e0 of each step is the linking edge of least
// frequent label.  Ties: lowest query vertex id.
void plan_order(const QueryGraph &q, const uint64_t *cand, const uint64_t *freq, int32_t nlabels, int32_t *order,
                int32_t *first) {
    const int k = q.k;
    double score[GSI_MAX_QUERY_VERTICES];
    auto fq = [&](int32_t l) -> double { return (l >= 0 && l < nlabels) ? (double)freq[l] : 0.0; };
    for (int u = 0; u < k; ++u) {
        int deg = 0;
        for (int w = 0; w < k; ++w) deg += q.elab[u][w] >= 0;
        score[u] = (double)cand[u] / (double)(deg > 0 ? deg : 1);
    }
    uint32_t matched = 0;
    for (int p = 0; p < k; ++p) {
        int best = -1;
        for (int u = 0; u < k; ++u) {
            if ((matched >> u) & 1u) continue;
            if (p > 0) {
                bool linked = false;
                for (int w = 0; w < k; ++w) linked |= ((matched >> w) & 1u) && q.elab[u][w] >= 0;
                if (!linked) continue;
            }
            if (best < 0 || score[u] < score[best]) best = u;
        }
        order[p] = best;
        first[p] = -1;
        if (p > 0) {
            double bf = 0;
            for (int w = 0; w < k; ++w) {
                if (!((matched >> w) & 1u) || q.elab[best][w] < 0) continue;
                double f = fq(q.elab[best][w]);
                if (first[p] < 0 || f < bf) { first[p] = w; bf = f; }
            }
        }
        matched |= 1u << best;
        for (int w = 0; w < k; ++w)
            if (q.elab[best][w] >= 0) score[w] *= fq(q.elab[best][w]);
    }
}

// JoinStep for position p (t = p columns), given the order and e0 choice.
void make_steps(const QueryGraph &q, const int32_t *order, const int32_t *first, const int32_t *ranks,
                std::vector<JoinStep> &steps) {
    const int k = q.k;
    int pos[GSI_MAX_QUERY_VERTICES];
    for (int p = 0; p < k; ++p) pos[order[p]] = p;
    steps.assign(k, JoinStep());
    for (int p = 1; p < k; ++p) {
        JoinStep &s = steps[p];
        s.t = p;
        s.d = 0;
        int u = order[p];
        s.ulab = ranks[u];
        s.col[s.d] = pos[first[p]];
        s.lab[s.d] = q.elab[u][first[p]];
        ++s.d;
        for (int c = 0; c < p; ++c) {
            int w = order[c];
            if (w == first[p] || q.elab[u][w] < 0) continue;
            s.col[s.d] = c;
            s.lab[s.d] = q.elab[u][w];
            ++s.d;
        }
        for (int c = 0; c <= p; ++c) s.perm[c] = (p == k - 1) ? order[c] : c;
        // only a column whose query vertex carries u's label can hold u's
        // image, so the set subtraction tests those columns alone
        s.inj = 0;
        for (int c = 0; c < p; ++c)
            if (ranks[order[c]] == ranks[u]) s.inj |= 1u << c;
    }
}

// -------------------------------------------------------------- timing
// Events are recycled through a per-thread pool: creating and destroying two
// events per launch would cost more host time than the launches themselves.
static thread_local std::vector<cudaEvent_t> t_event_pool;

static cudaEvent_t pooled_event() {
    if (!t_event_pool.empty()) {
        cudaEvent_t e = t_event_pool.back();
        t_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Timer::begin(int kind) {
    if (!on) return;
    Rec r;
    r.kind = kind;
    r.a = pooled_event();
    r.b = pooled_event();
    cudaEventRecord(r.a, st);
    recs.push_back(r);
}
void Timer::end() {
    if (!on || recs.empty()) return;
    cudaEventRecord(recs.back().b, st);
}
void Timer::resolve(gsi_stats *s) {
    for (auto &r : recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        if (s) {
            if (r.kind == 0) { s->filter_ms += ms; s->filter_launches++; }
            else if (r.kind == 1) { s->join_ms += ms; s->join_launches++; }
            else { s->other_ms += ms; s->other_launches++; }
        }
        t_event_pool.push_back(r.a);
        t_event_pool.push_back(r.b);
    }
    recs.clear();
}

// ----------------------------------------------------------------- driver
// First device-driven arena of a query.  Reserving an arena near the whole
// default budget (a large share of HBM) from the stream-ordered pool costs
// milliseconds per query; arenas up to tens of GB cost well under one.
constexpr uint64_t DEVICE_ARENA_START = 16ull << 30;

static std::atomic<uint64_t> g_total_mem[64];
static std::atomic<uint64_t> g_held[64];

uint64_t device_total_mem(int dev) {
    if (dev < 0 || dev >= 64) return 0;
    uint64_t t = g_total_mem[dev].load();
    if (!t) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        t = tot;
        g_total_mem[dev].store(t);
    }
    return t;
}

bool hold_region(int dev, uint64_t bytes) {
    if (dev < 0 || dev >= 64) return false;
    const uint64_t limit = device_total_mem(dev) / 4;
    uint64_t cur = g_held[dev].load();
    while (cur + bytes <= limit)
        if (g_held[dev].compare_exchange_weak(cur, cur + bytes)) return true;
    return false;
}

void release_region(int dev, uint64_t bytes) {
    if (dev >= 0 && dev < 64) g_held[dev].fetch_sub(bytes);
}

static gsi_status dalloc(Exec &x, void **p, uint64_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, x.st);
    if (e != cudaSuccess) {
        set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        return GSI_ENOMEM;
    }
    return GSI_OK;
}

static gsi_status read_u64(Exec &x, const void *dptr, uint64_t *val) {
    GSI_CUDA_TRY(cudaMemcpyAsync(x.h_pinned, dptr, 8, cudaMemcpyDeviceToHost, x.st));
    GSI_CUDA_TRY(cudaStreamSynchronize(x.st));
    *val = x.h_pinned[0];
    return GSI_OK;
}

gsi_status Exec::add_chunk(int32_t *rows, uint64_t nrows, uint64_t alloc_rows) {
    if (nrows == 0) {
        cudaFreeAsync(rows, st);
        return GSI_OK;
    }
    if (alloc_rows > 2 * nrows + 1024) {   // shrink a loose Prealloc bound
        int32_t *tight = nullptr;
        uint64_t bytes = nrows * (uint64_t)k * 4;
        GSI_TRY(dalloc(*this, (void **)&tight, bytes));
        GSI_CUDA_TRY(cudaMemcpyAsync(tight, rows, bytes, cudaMemcpyDeviceToDevice, st));
        cudaFreeAsync(rows, st);
        rows = tight;
    }
    res->chunks.push_back({rows, nrows});
    res->materialised += nrows;
    return GSI_OK;
}

// Extend the t-column table M (R rows) by position t, then recurse to the
// last position.  Memory-bounded: when the step's buffers would exceed the
// budget, M is halved by rows and each half is finished depth-first.
gsi_status Exec::run(int t, const int32_t *M, uint64_t R) {
    if (R == 0) return GSI_OK;
    const JoinStep &s = steps[t];
    const bool last = (t + 1 == k);
    const uint64_t fbytes = 8 * (R + 1) + 8 * (uint64_t)join_scan_scratch(R);
    auto split = [&]() -> gsi_status {
        uint64_t h = R / 2;
        GSI_TRY(run(t, M, h));
        return run(t, M + h * (uint64_t)t, R - h);
    };
    if (live + fbytes > budget) {
        if (R > 1) return split();
        set_error("memory budget cannot hold a one-row tile");
        return GSI_ENOMEM;
    }
    uint64_t *F = nullptr, *scr = nullptr;
    GSI_TRY(dalloc(*this, (void **)&F, 8 * (R + 1)));
    GSI_TRY(dalloc(*this, (void **)&scr, 8 * (uint64_t)join_scan_scratch(R)));
    tm.begin(2);
    gsi_status rc = launch_join_scan(g, M, R, s, F, scr, st);
    tm.end();
    kernels += 3;
    uint64_t total = 0;
    if (rc == GSI_OK) rc = read_u64(*this, F + R, &total);
    cudaFreeAsync(scr, st);
    if (rc != GSI_OK) {
        cudaFreeAsync(F, st);
        return rc;
    }
    const uint64_t sumcap = total - (uint64_t)JOIN_ROW_WEIGHT * R;
    uint64_t out_rows = sumcap;
    int count_mode = 0;
    if (last) {
        uint64_t room = row_cap ? (res->materialised >= row_cap ? 0 : row_cap - res->materialised) : sumcap;
        out_rows = count_only ? 0 : std::min(sumcap, room);
        count_mode = out_rows == 0;
    }
    const uint64_t ntiles = join_tiles(total);
    const uint64_t obytes = out_rows * (uint64_t)(t + 1) * 4;
    const uint64_t need = 8 * (R + 1) + 8 * (ntiles + 1) + obytes;
    if (live + need > budget) {
        cudaFreeAsync(F, st);
        if (R > 1) return split();
        set_error("memory budget cannot hold a one-row tile");
        return GSI_ENOMEM;
    }
    int64_t *part = nullptr;
    int32_t *out = nullptr;
    rc = dalloc(*this, (void **)&part, 8 * (ntiles + 1));
    if (rc == GSI_OK) rc = dalloc(*this, (void **)&out, obytes);
    if (rc != GSI_OK) {
        cudaFreeAsync(F, st);
        if (part) cudaFreeAsync(part, st);
        return rc;
    }
    live += need;
    peak = std::max(peak, live);
    ++tiles;
    if (cudaMemsetAsync(d_scalars, 0, 8, st) != cudaSuccess) rc = GSI_ECUDA;
    if (rc == GSI_OK) {
        tm.begin(2);
        rc = launch_partition(F, R, total, part, st);
        tm.end();
        kernels += total > 0;
    }
    if (rc == GSI_OK) {
        tm.begin(1);
        rc = launch_join(g, M, R, s, F, total, part, cand(s, t), out, out_rows, d_scalars, count_mode,
                         stats ? d_scalars + 1 : nullptr, st);
        tm.end();
        kernels += total > 0;
    }
    uint64_t cnt = 0;
    if (rc == GSI_OK) rc = read_u64(*this, d_scalars, &cnt);
    cudaFreeAsync(F, st);
    cudaFreeAsync(part, st);
    live -= 8 * (R + 1) + 8 * (ntiles + 1);
    if (rc != GSI_OK) {
        cudaFreeAsync(out, st);
        live -= obytes;
        return rc;
    }
    if (last) {
        res->count += cnt;
        live -= obytes;
        if (count_mode) {
            cudaFreeAsync(out, st);
            return GSI_OK;
        }
        return add_chunk(out, std::min(cnt, out_rows), out_rows);
    }
    rc = run(t + 1, out, cnt);
    cudaFreeAsync(out, st);
    live -= obytes;
    return rc;
}


// Device-driven execution of the whole join: one arena per query (a scratch
// region and two table regions used in turn), every step's sizes computed on
// the device, no host wait until the end.  The final table's region is handed
// to the result when it is well used, or its rows are copied to a tight buffer.
gsi_status Exec::run_device(uint64_t arena_bytes, bool *overflow, bool *no_memory) {
    *overflow = false;
    *no_memory = false;
    const uint64_t B = arena_bytes;
    const uint64_t align = 256;
    // a third each: scratch (16 bytes per input row: offsets and bound
    // records) and two table regions (a row of t + 1 >= 4 columns needs as
    // much table space as its successor step needs scratch)
    const uint64_t s_bytes = (B / 3) / align * align;
    const uint64_t t_bytes = ((B - s_bytes) / 2) / align * align;
    if (s_bytes < (1 << 16) || t_bytes < (uint64_t)g->n * 4 + 1024) {
        *overflow = true;
        *no_memory = true;
        return GSI_OK;
    }
    uint64_t *S = nullptr, *memo = nullptr;
    int32_t *reg[2] = {nullptr, nullptr};
    unsigned char *ctl = nullptr;
    const uint64_t memo_bytes = nodedup ? 0 : (uint64_t)query_memo_tables(steps, k) * (uint64_t)g->n * 8;
    const size_t ctl_bytes = (join_args_size() * (size_t)k + 255) / 256 * 256 +
                             (sizeof(DStep) * (size_t)k + 255) / 256 * 256 + 256 + 8 * (size_t)QUERY_MAX_CTAS;
    gsi_status rc = dalloc(*this, (void **)&S, s_bytes);
    if (rc == GSI_OK) rc = dalloc(*this, (void **)&reg[0], t_bytes);
    if (rc == GSI_OK) rc = dalloc(*this, (void **)&reg[1], t_bytes);
    if (rc == GSI_OK) rc = dalloc(*this, (void **)&ctl, ctl_bytes);
    if (rc == GSI_OK && memo_bytes) rc = dalloc(*this, (void **)&memo, memo_bytes);
    auto release = [&]() {
        if (memo) cudaFreeAsync(memo, st);
        if (S) cudaFreeAsync(S, st);
        if (reg[0]) cudaFreeAsync(reg[0], st);
        if (reg[1]) cudaFreeAsync(reg[1], st);
        if (ctl) cudaFreeAsync(ctl, st);
    };
    if (rc != GSI_OK) {
        release();
        (void)cudaGetLastError();
        *overflow = true;              // could not reserve the arena: use the splitting path
        *no_memory = true;
        return GSI_OK;
    }
    peak = std::max(peak, s_bytes + 2 * t_bytes);
    // control block: [step configs][step records][barrier/status][per-CTA sums]
    unsigned char *p = ctl;
    void *cfg_dev = p;
    p += (join_args_size() * (size_t)k + 255) / 256 * 256;
    DStep *dst = reinterpret_cast<DStep *>(p);
    p += (sizeof(DStep) * (size_t)k + 255) / 256 * 256;
    QueryCtl *qc = reinterpret_cast<QueryCtl *>(p);
    p += 256;
    unsigned long long *bsum = reinterpret_cast<unsigned long long *>(p);
    // configurations, step records and zeroed control words staged in pinned
    // memory in the control block's layout: one upload, no staging copies
    const size_t up_bytes = (size_t)(p - ctl);
    if (up_bytes > h_stage_bytes) {
        release();
        set_error("device-driven join: control block larger than the staging buffer");
        return GSI_EINVAL;
    }
    unsigned long long *jstats = stats ? d_scalars + 1 : nullptr;
    size_t smem = 0;
    rc = query_coop_configs(g, steps, k, bitmaps, order, count_only, jstats, memo, nodedup, h_stage, &smem);
    if (rc != GSI_OK) {
        release();
        return rc;
    }
    DStep *hs = reinterpret_cast<DStep *>(h_stage + (reinterpret_cast<unsigned char *>(dst) - ctl));
    std::memset(hs, 0, sizeof(DStep) * (size_t)k);
    std::memset(h_stage + (reinterpret_cast<unsigned char *>(qc) - ctl), 0, 256);
    for (int t = 1; t < k; ++t) {
        DStep &h = hs[t];
        h.M = reg[(t - 1) & 1];
        h.out = reg[t & 1];
        h.out_bytes = t_bytes;
        const bool last = t == k - 1;
        h.row_cap = last ? row_cap : 0;
        h.count_only = last ? count_only : 0;
        h.S = S;
        h.S_words = s_bytes / 8;
        h.t = t;
    }
    rc = GSI_OK;
    if (memo_bytes && cudaMemsetAsync(memo, 0, memo_bytes, st) != cudaSuccess) {
        set_error("device-driven join: clearing the sub-list memo failed");
        rc = GSI_ECUDA;
    }
    if (rc == GSI_OK && cudaMemcpyAsync(ctl, h_stage, up_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_error("device-driven join: control upload failed");
        rc = GSI_ECUDA;
    }
    int grid = 0;
    if (rc == GSI_OK) {
        tm.begin(1);
        rc = launch_query_coop(g, k, bitmaps + (uint64_t)order[0] * (uint64_t)g->nwords, smem, cfg_dev, dst, qc, bsum,
                               &grid, listwise && stats, st);
        tm.end();
        kernels += 1;
        tiles += (uint64_t)(k - 1);
    }
    // read back: status, and the final count / capacity
    uint64_t fin[3] = {0, 0, 0};
    if (rc == GSI_OK) {
        if (cudaMemcpyAsync(h_pinned, &qc->fail, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(h_pinned + 1, &dst[k - 1].count, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(h_pinned + 2, &dst[k - 1].out_cap, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (stats && cudaMemcpyAsync(h_pinned + 3, d_scalars + 1, 24, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("device-driven join: kernel or readback failed");
            rc = GSI_ECUDA;
        }
        fin[0] = h_pinned[0] & 0xffffffffu;
        fin[1] = h_pinned[1];
        fin[2] = h_pinned[2];
        if (rc == GSI_OK && stats && fin[0] == 0) {   // the join's counters, read with the status
            join_bytes = h_pinned[3];
            join_items = h_pinned[4];
            join_bytes_listwise = h_pinned[5];
            stats_read = true;
        }
    }
    if (rc == GSI_OK && (fin[0] & 4u)) {
        release();
        set_error("device-driven join: a grid barrier wait ran past its limit");
        return GSI_ETIMEOUT;
    }
    if (rc != GSI_OK || fin[0] != 0) {
        release();
        if (rc == GSI_OK) *overflow = true;
        return rc;
    }
    const uint64_t count = fin[1];
    // the last table must hold every row asked for (all, or up to the row cap)
    const uint64_t need = count_only ? 0 : (row_cap ? std::min(count, row_cap) : count);
    if (need > fin[2]) {
        release();
        *overflow = true;
        return GSI_OK;
    }
    const uint64_t rows = std::min(count, fin[2]);
    int32_t *final_reg = reg[(k - 1) & 1];
    res->count += count;
    if (rows > 0) {
        const uint64_t bytes = rows * (uint64_t)k * 4;
        // the result keeps the region when its rows fill a quarter of it, or
        // while the device's allowance for held regions lasts; otherwise (and
        // always when asked for tight rows) the rows move to a tight buffer
        const bool big = bytes * 4 >= t_bytes;
        if (!tight_rows && (big || hold_region(g->device, t_bytes))) {
            gsi_result::Chunk ch{final_reg, rows};
            ch.held = big ? 0 : t_bytes;
            res->chunks.push_back(ch);
            res->materialised += rows;
            reg[(k - 1) & 1] = nullptr;
        } else {
            int32_t *tight = nullptr;
            rc = dalloc(*this, (void **)&tight, bytes);
            if (rc == GSI_OK && cudaMemcpyAsync(tight, final_reg, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                set_error("device-driven join: result copy failed");
                rc = GSI_ECUDA;
            }
            if (rc == GSI_OK) {
                res->chunks.push_back({tight, rows});
                res->materialised += rows;
            } else if (tight) {
                cudaFreeAsync(tight, st);
            }
        }
    }
    release();
    return rc;
}

gsi_status plan_for_batch(gsi_graph *g, BatchPlan &p, const uint64_t *cand_counts, const int32_t *ranks) {
    int32_t first[GSI_MAX_QUERY_VERTICES];
    plan_order(p.q, cand_counts, g->freq.data(), g->L, p.order, first);
    make_steps(p.q, p.order, first, ranks, p.steps);
    p.seed_count = cand_counts[p.order[0]];
    return GSI_OK;
}

const uint32_t *Exec::cand(const JoinStep &s, int t) const {
    (void)s;
    return bitmaps + (uint64_t)order[t] * (uint64_t)g->nwords;
}

gsi_status run_query(gsi_graph *g, const QueryGraph &q, const gsi_query_opts &o, gsi_result **out) {
    GSI_TRY(prepare_device(g->device));
    std::unique_ptr<gsi_result> res(new gsi_result());
    res->k = q.k;
    res->device = g->device;
    res->stream = (cudaStream_t)o.stream;
    res->own_stream = true;
    Exec x;
    x.g = g;
    x.k = q.k;
    x.st = (cudaStream_t)o.stream;
    x.row_cap = o.row_cap;
    x.count_only = o.count_only;
    x.stats = o.stats;
    x.listwise = o.listwise_bytes != 0;
    x.nodedup = o.no_dedup != 0;
    x.tight_rows = o.tight_rows != 0;
    x.res = res.get();
    x.tm.on = o.stats != nullptr;
    x.tm.st = x.st;
    if (o.mem_budget) {
        x.budget = o.mem_budget;
    } else {
        // a fixed share of the device (not of the momentarily free memory, which
        // excludes blocks the stream-ordered pool keeps cached for reuse); the
        // device's total is looked up once
        const uint64_t totm = device_total_mem(g->device);
        if (!totm) {
            set_error("query: device memory size unavailable");
            return GSI_ECUDA;
        }
        x.budget = (uint64_t)(0.4 * (double)totm);
    }
    // a query edge label that no data edge carries: no embeddings
    for (int e = 0; e < q.qm; ++e)
        if (q.lab[e] >= g->L || g->freq[q.lab[e]] == 0) {
            *out = res.release();
            return GSI_OK;
        }
    if (q.k > 1 && g->m == 0) {
        *out = res.release();
        return GSI_OK;
    }
    // a query vertex label that no data vertex carries: no embeddings
    int32_t ranks[GSI_MAX_QUERY_VERTICES];
    for (int u = 0; u < q.k; ++u) {
        ranks[u] = g->label_rank(q.vlab[u]);
        if (ranks[u] < 0) {
            *out = res.release();
            return GSI_OK;
        }
    }

    QuerySig qs;
    const bool hom = o.semantics == GSI_HOMOMORPHISM;
    query_signatures(q.vl.data(), q.k, q.src.data(), q.dst.data(), q.lab.data(), q.qm, &qs, hom);
    const uint64_t bm_words = (uint64_t)q.k * (uint64_t)g->nwords;
    // per-thread pinned staging: small readbacks first, then the upload area
    // of the device-driven control block (cudaFreeHost would synchronise the
    // whole device, so the buffer lives as long as the thread).  Every use is
    // complete before run_query returns (the stream is synchronised).
    static thread_local unsigned char *t_pinned = nullptr;
    constexpr size_t PINNED_READ = 4096, PINNED_STAGE = 60 * 1024;
    if (!t_pinned) GSI_CUDA_TRY(cudaMallocHost(&t_pinned, PINNED_READ + PINNED_STAGE));
    x.h_pinned = reinterpret_cast<uint64_t *>(t_pinned);
    x.h_stage = t_pinned + PINNED_READ;
    x.h_stage_bytes = PINNED_STAGE;
    unsigned long long *d_counts = nullptr;
    gsi_status rc = dalloc(x, (void **)&x.bitmaps, bm_words * 4);
    if (rc == GSI_OK) rc = dalloc(x, (void **)&d_counts, 8 * GSI_MAX_QUERY_VERTICES + 32);
    if (rc == GSI_OK) {
        x.d_scalars = d_counts + GSI_MAX_QUERY_VERTICES;
        if (cudaMemsetAsync(x.d_scalars, 0, 32, x.st) != cudaSuccess) {
            set_error("query: clearing the counters failed");
            rc = GSI_ECUDA;
        }
    }
    if (rc != GSI_OK) {                     // nothing was launched: release what was reserved
        if (x.bitmaps) cudaFreeAsync(x.bitmaps, x.st);
        if (d_counts) cudaFreeAsync(d_counts, x.st);
        return rc;
    }

    x.tm.begin(0);
    rc = launch_filter(g, qs, x.bitmaps, d_counts, x.st);
    x.tm.end();
    x.kernels += 1;
    uint64_t cand_h[GSI_MAX_QUERY_VERTICES] = {0};
    if (rc == GSI_OK) {
        if (cudaMemcpyAsync(x.h_pinned, d_counts, 8 * (size_t)q.k, cudaMemcpyDeviceToHost, x.st) != cudaSuccess ||
            cudaStreamSynchronize(x.st) != cudaSuccess) {
            set_error("filter: readback failed");
            rc = GSI_ECUDA;
        } else {
            for (int u = 0; u < q.k; ++u) cand_h[u] = x.h_pinned[u];
        }
    }
    bool empty = false;
    for (int u = 0; u < q.k; ++u) empty |= cand_h[u] == 0;

    int32_t order[GSI_MAX_QUERY_VERTICES], first[GSI_MAX_QUERY_VERTICES];
    if (rc == GSI_OK && !empty) {
        if (o.order) {
            uint32_t seen = 0;
            for (int p = 0; p < q.k && rc == GSI_OK; ++p) {
                int u = o.order[p];
                bool ok = u >= 0 && u < q.k && !((seen >> u) & 1u);
                if (ok && p > 0) {
                    bool linked = false;
                    for (int w = 0; w < q.k; ++w) linked |= ((seen >> w) & 1u) && q.elab[u][w] >= 0;
                    ok = linked;
                }
                if (!ok) {
                    set_error("query: forced order is not a connected permutation");
                    rc = GSI_EINVAL;
                    break;
                }
                seen |= 1u << u;
                order[p] = u;
                first[p] = -1;
                if (p > 0) {
                    double bf = 0;
                    for (int w = 0; w < q.k; ++w) {
                        if (!((seen >> w) & 1u) || w == u || q.elab[u][w] < 0) continue;
                        double f = (double)g->freq[q.elab[u][w]];
                        if (first[p] < 0 || f < bf) { first[p] = w; bf = f; }
                    }
                }
            }
        } else {
            plan_order(q, cand_h, g->freq.data(), g->L, order, first);
        }
    }
    if (rc == GSI_OK && !empty) {
        for (int p = 0; p < q.k; ++p) x.order[p] = order[p];
        make_steps(q, order, first, ranks, x.steps);
        for (JoinStep &js : x.steps) js.hom = hom ? 1 : 0;
        // device-driven path first; the host-driven splitting path on overflow
        bool overflow = true;
        if (!o.host_driven && q.k > 1) {
            // arenas of 16 GiB, then x4 per overflow, up to the budget
            uint64_t arena = std::min<uint64_t>(x.budget, DEVICE_ARENA_START);
            for (;;) {
                bool no_memory = false;
                rc = x.run_device(arena, &overflow, &no_memory);
                if (rc != GSI_OK || !overflow || no_memory || arena >= x.budget) break;
                arena = std::min<uint64_t>(x.budget, arena * 4);
            }
        }
        x.fell_back = overflow;
        const uint64_t R0 = cand_h[order[0]];
        int32_t *M0 = nullptr;
        if (rc == GSI_OK && overflow) {
            // seed: M = C(u_first) as a one-column table (Alg. 2)
            uint32_t *sscr = nullptr;
            rc = dalloc(x, (void **)&M0, R0 * 4);
            if (rc == GSI_OK) rc = dalloc(x, (void **)&sscr, 4 * (uint64_t)seed_scratch_words(g));
            if (rc == GSI_OK) {
                x.tm.begin(2);
                rc = launch_seed(g, x.bitmaps + (uint64_t)order[0] * g->nwords, M0, sscr, x.st);
                x.tm.end();
                x.kernels += 3;
            }
            if (sscr) cudaFreeAsync(sscr, x.st);
            if (rc == GSI_OK) {
                x.live = R0 * 4;
                if (q.k == 1) {
                    res->count = R0;
                    uint64_t keep = x.count_only ? 0 : (x.row_cap ? std::min(R0, x.row_cap) : R0);
                    if (keep) {
                        rc = x.add_chunk(M0, keep, R0);
                        M0 = nullptr;
                    }
                } else {
                    rc = x.run(1, M0, R0);
                }
            }
        }
        if (M0) cudaFreeAsync(M0, x.st);
    }
    if (x.stats && rc == GSI_OK && !(x.stats_read && !x.fell_back)) {
        // algorithmic bytes and candidates counted by the join kernels
        if (cudaMemcpyAsync(x.h_pinned, x.d_scalars + 1, 24, cudaMemcpyDeviceToHost, x.st) == cudaSuccess &&
            cudaStreamSynchronize(x.st) == cudaSuccess) {
            x.join_bytes = x.h_pinned[0];
            x.join_items = x.h_pinned[1];
            x.join_bytes_listwise = x.h_pinned[2];
        }
    }
    cudaFreeAsync(x.bitmaps, x.st);
    cudaFreeAsync(d_counts, x.st);
    cudaError_t se = cudaStreamSynchronize(x.st);
    if (rc == GSI_OK && se != cudaSuccess) {
        set_error(std::string("query: ") + cudaGetErrorString(se));
        rc = GSI_ECUDA;
    }
    if (x.stats) {
        gsi_stats *s = x.stats;
        x.tm.resolve(s);
        s->k = q.k;
        for (int u = 0; u < q.k; ++u) s->cand[u] = cand_h[u];
        for (int p = 0; p < q.k; ++p) s->order[p] = (rc == GSI_OK && !empty) ? order[p] : -1;
        s->tiles += x.tiles;
        s->peak_bytes = std::max<uint64_t>(s->peak_bytes, x.peak);
        s->filter_bytes += filter_alg_bytes(g, std::vector<int32_t>(q.vlab, q.vlab + q.k));
        s->join_bytes += x.join_bytes;
        s->join_items += x.join_items;
        s->join_bytes_listwise += x.join_bytes_listwise;
        s->kernels += x.kernels;
        s->host_driven += (rc == GSI_OK && !empty && x.fell_back) ? 1 : 0;
    }
    if (rc != GSI_OK) return rc;
    *out = res.release();
    return GSI_OK;
}

}  // namespace gsi

extern "C" const char *gsi_last_error(void) { return gsi::last_error(); }

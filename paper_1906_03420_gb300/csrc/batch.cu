// Batched execution: many queries' joins in one persistent launch.
//
// Work items are (query, range of words of the query's seed bitmap C(u_first))
// pairs on a shared queue.  A CTA takes an item, seeds its table with the set
// bits of its word range, and runs every join step of the query on those rows
// depth-first inside its own slice of the batch arena (a scratch region and
// two table regions used in turn), with CTA-local scans and CTA-local
// survivor counters: items never wait on one another.  The final rows are
// appended to a result arena shared by all items (one atomic reservation per
// item); each item records where its rows went.  An item whose table does not
// fit its slice, or whose rows do not fit the result arena, marks its query
// failed; the host runs failed queries again on the plain path.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "join_tile.cuh"
#include "runtime.h"

namespace gsi {
namespace {

constexpr int BNT = JOIN_NT;
constexpr int BVT = JOIN_VT;
constexpr int BNV = BNT * BVT;

struct BatchQuery {
    const uint32_t *seed_bm;       // bitmap of C(u_first)
    int32_t k;
    int32_t count_only;
    unsigned status;               // 1 = failed (table or result arena overflow)
    unsigned pad;
    unsigned long long count;      // embeddings (summed over items)
};

struct BatchItem {
    int32_t q;
    int32_t pad;
    int64_t word_lo, word_hi;
};

struct BatchRec {
    unsigned long long off;        // int32 offset of the item's rows in the result arena
    unsigned long long rows;
};

struct BatchArgs {
    const JoinArgs *cfgs;          // [q * 32 + t]
    BatchQuery *queries;
    const BatchItem *items;
    BatchRec *recs;
    int64_t nitems;
    unsigned long long *next_item;
    int32_t *result;               // result arena
    unsigned long long result_cap; // int32 elements
    unsigned long long *result_used;
    unsigned char *arena;          // per-CTA slices
    uint64_t slice_bytes, s_bytes, t_bytes;
    uint64_t item_rows;            // an item whose table grows past this fails over (0 = region size)
};

__global__ void __launch_bounds__(BNT) k_batch(const __grid_constant__ BatchArgs b) {
    __shared__ unsigned long long wt[BNT / 32];
    __shared__ long long item_s;
    __shared__ unsigned long long cnt_s, off_s;
    __shared__ int fail_s;
    unsigned char *slice = b.arena + (uint64_t)blockIdx.x * b.slice_bytes;
    uint64_t *S = reinterpret_cast<uint64_t *>(slice);
    int32_t *reg[2] = {reinterpret_cast<int32_t *>(slice + b.s_bytes),
                       reinterpret_cast<int32_t *>(slice + b.s_bytes + b.t_bytes)};
    const uint64_t S_words = b.s_bytes / 8;
    const uint64_t W = (uint64_t)JOIN_ROW_WEIGHT;

    for (;;) {
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(b.next_item, 1ull);
        __syncthreads();
        const long long item = item_s;
        if (item >= b.nitems) return;
        const BatchItem it = b.items[item];
        BatchQuery *bq = b.queries + it.q;
        const int k = bq->k;
        // ---- seed: set bits of the item's words, ascending
        uint64_t R = 0;
        {
            unsigned long long run = 0;
            for (int64_t base = it.word_lo; base < it.word_hi; base += BNT) {
                const int64_t i = base + threadIdx.x;
                const uint32_t w = i < it.word_hi ? bq->seed_bm[i] : 0u;
                unsigned long long tot;
                unsigned long long pos = block_exclusive_scan<BNT, unsigned long long>(__popc(w), wt, &tot) + run;
                uint32_t x = w;
                while (x) {
                    reg[0][pos++] = (int32_t)(i * 32 + (int64_t)(__ffs(x) - 1));
                    x &= x - 1;
                }
                run += tot;
            }
            R = run;
        }
        __syncthreads();               // step 1 reads seeds written by other threads
        int cur = 0;
        bool failed = false;
        uint64_t cap = 0;
        for (int t = 1; t < k && R > 0; ++t) {
            const JoinArgs &a = b.cfgs[(size_t)it.q * GSI_MAX_QUERY_VERTICES + t];
            const int32_t *M = reg[cur];
            int32_t *out = reg[cur ^ 1];
            if ((R + 1) * 8 + R * 4 + 64 > S_words * 8) { failed = true; break; }
            uint64_t *F = S;
            uint32_t *caps = reinterpret_cast<uint32_t *>(S + S_words) - R;
            // bounds and slot offsets (CTA-local scan)
            unsigned long long run = 0;
            for (uint64_t base = 0; base < R; base += BNT) {
                const uint64_t i = base + threadIdx.x;
                unsigned long long v = 0;
                if (i < R) {
                    const uint32_t c = row_bound(a.s, M + i * (uint64_t)a.s.t, a.off, a.cl);
                    caps[i] = c;
                    v = (unsigned long long)c + W;
                }
                unsigned long long tot;
                const unsigned long long ex = block_exclusive_scan<BNT, unsigned long long>(v, wt, &tot) + run;
                if (i < R) F[i] = ex;
                run += tot;
            }
            const uint64_t total = run;
            if (threadIdx.x == 0) {
                F[R] = total;
                cnt_s = 0;
            }
            const bool last = t == k - 1;
            cap = b.t_bytes / (4ull * (uint64_t)(t + 1));
            if (last && bq->count_only) cap = 0;
            __syncthreads();
            // tiles in order; each tile spans at most BNV/W + 1 rows past its first
            const uint64_t ntiles = (total + BNV - 1) / BNV;
            int64_t r_lo = 0;
            const uint64_t span = BNV / W + 1;
            for (uint64_t tile = 0; tile < ntiles; ++tile) {
                const uint64_t s_next = min((tile + 1) * (uint64_t)BNV, total);
                const uint64_t lim = min((uint64_t)R - (uint64_t)r_lo, span);
                unsigned long long c = 0;
                for (uint64_t j = threadIdx.x; j <= lim; j += BNT) c += F[r_lo + j] <= s_next;
                c = block_sum<BNT, unsigned long long>(c, wt);
                const int64_t r_next = r_lo + (int64_t)c - 1;
                join_tile<BNT, BVT>(a, M, (int64_t)R, F, total, r_lo, r_next, out, cap, &cnt_s, tile);
                r_lo = r_next;
            }
            __syncthreads();
            const uint64_t cnt = cnt_s;
            if (!last && cnt > cap) { failed = true; break; }
            if (b.item_rows && cnt > b.item_rows) { failed = true; break; }
            R = cnt;
            cur ^= 1;
        }
        if (k == 1) cap = bq->count_only ? 0 : b.t_bytes / 4;
        // the final table must also have fit (rows past the region are lost)
        if (!failed && !bq->count_only && R > cap) failed = true;
        // ---- final rows to the result arena
        const uint64_t rows = failed ? 0 : min(R, cap);
        if (threadIdx.x == 0) {
            fail_s = failed;
            off_s = 0;
            if (!failed && rows > 0) {
                const unsigned long long need = rows * (unsigned long long)k;
                const unsigned long long o = atomicAdd(b.result_used, need);
                if (o + need > b.result_cap) fail_s = 1;
                else off_s = o;
            }
            if (fail_s) atomicOr(&bq->status, 1u);
            else atomicAdd(&bq->count, (unsigned long long)R);
            b.recs[item].off = off_s;
            b.recs[item].rows = fail_s ? 0 : rows;
        }
        __syncthreads();
        if (!fail_s && rows > 0) {
            const int32_t *src = reg[cur];
            int32_t *dst = b.result + off_s;
            const uint64_t n = rows * (uint64_t)k;
            for (uint64_t i = threadIdx.x; i < n; i += BNT) dst[i] = src[i];
        }
        __syncthreads();
    }
}

}  // namespace

// Per-query plan for a batch: the host-side part of run_query (filter counts
// already known), producing the steps of one query.
gsi_status batch_run_device(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &o,
                            uint64_t budget, cudaStream_t st, gsi_stats *stats, BatchWorkspace *ws) {
    const int nq = (int)plans.size();
    if (nq == 0) return GSI_OK;
    // device counters of algorithmic bytes and candidates (only with stats)
    unsigned long long *dstats = nullptr;
    if (stats) {
        GSI_CUDA_TRY(cudaMallocAsync(&dstats, 16, st));
        GSI_CUDA_TRY(cudaMemsetAsync(dstats, 0, 16, st));
    }
    // configs, queries, items
    std::vector<JoinArgs> cfg((size_t)nq * GSI_MAX_QUERY_VERTICES);
    std::vector<BatchQuery> bqs((size_t)nq);
    std::vector<BatchItem> items;
    size_t sm = join_smem(JOIN_NV / JOIN_ROW_WEIGHT + 2, 1, 1);
    for (int i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        if (!p.active) continue;
        for (int t = 1; t < p.k; ++t)
            sm = std::max(sm, join_smem(JOIN_NV / JOIN_ROW_WEIGHT + 2, p.steps[t].t, p.steps[t].d));
    }
    if (sm > 200 * 1024) {
        set_error("batch: shared memory need exceeds 200 KB");
        return GSI_EINVAL;
    }
    int dev = 0, nsm = 152, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    GSI_CUDA_TRY(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    GSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BNT, sm));
    if (per_sm < 1) {
        set_error("batch: kernel does not fit on an SM");
        return GSI_EINVAL;
    }
    // memory: result arena 40%, per-CTA slices 60% (scratch 20%, two tables
    // 40% each); fewer CTAs when the budget would make slices too small
    const uint64_t align = 256, min_table = 1ull << 20;
    const uint64_t result_bytes = ws ? ws->result_bytes : (budget * 2 / 5) / align * align;
    const uint64_t slices_bytes = ws ? ws->arena_bytes : budget - result_bytes;
    int grid = nsm * per_sm;
    while (grid > 1 && (slices_bytes / (uint64_t)grid) * 2 / 5 < min_table) grid /= 2;
    const uint64_t slice = (slices_bytes / (uint64_t)grid) / align * align;
    const uint64_t s_bytes = (slice / 5) / align * align;
    const uint64_t t_bytes = ((slice - s_bytes) / 2) / align * align;
    if (t_bytes < min_table) {
        for (BatchPlan &p : plans)                        // too small for any slice: all on the plain path
            if (p.active) p.failed = true;
        return GSI_OK;
    }
    // seed words per item: at most one table region of seeds
    const uint64_t max_words = std::max<uint64_t>(1, (t_bytes - 1024) / 128);
    for (int i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        std::memset(&bqs[i], 0, sizeof(BatchQuery));
        bqs[i].k = p.k;
        bqs[i].count_only = o.count_only;
        if (!p.active) continue;
        bqs[i].seed_bm = p.bitmaps + (uint64_t)p.order[0] * (uint64_t)g->nwords;
        for (int t = 1; t < p.k; ++t) {
            const int co = (t == p.k - 1) && o.count_only;
            cfg[(size_t)i * GSI_MAX_QUERY_VERTICES + t] =
                make_join_args(g, p.steps[t], p.bitmaps + (uint64_t)p.order[t] * (uint64_t)g->nwords, co, dstats);
        }
        // split the seed bitmap into word ranges holding about seeds_per_item
        // seeds each (and never more words than a table region can take)
        const uint64_t nw = (uint64_t)g->nwords;
        const uint64_t per = o.seeds_per_item > 0 ? (uint64_t)o.seeds_per_item : 32;
        uint64_t parts = std::max<uint64_t>((p.seed_count + per - 1) / per, (nw + max_words - 1) / max_words);
        if (parts < 1) parts = 1;
        if (parts > nw) parts = nw;
        for (uint64_t j = 0; j < parts; ++j) {
            BatchItem it;
            it.q = i;
            it.pad = 0;
            it.word_lo = (int64_t)(nw * j / parts);
            it.word_hi = (int64_t)(nw * (j + 1) / parts);
            if (it.word_hi > it.word_lo) items.push_back(it);
        }
    }
    const size_t ctl_bytes = sizeof(JoinArgs) * cfg.size() + sizeof(BatchQuery) * bqs.size() +
                             sizeof(BatchItem) * items.size() + sizeof(BatchRec) * items.size() + 64;
    unsigned char *ctl = nullptr, *arena = nullptr;
    int32_t *result = nullptr;
    auto free_all = [&]() {
        if (ctl) cudaFreeAsync(ctl, st);
        if (arena) cudaFreeAsync(arena, st);
        if (result) cudaFreeAsync(result, st);
    };
    auto free_all_ws = [&]() {
        if (ctl) cudaFreeAsync(ctl, st);
    };
    if (ws) {
        arena = ws->arena;
        result = ws->result;
    }
    if (cudaMallocAsync(&ctl, ctl_bytes, st) != cudaSuccess ||
        (!ws && cudaMallocAsync(&arena, slice * (uint64_t)grid, st) != cudaSuccess) ||
        (!ws && cudaMallocAsync(&result, result_bytes, st) != cudaSuccess)) {
        if (ws) {
            arena = nullptr;
            result = nullptr;
        }
        free_all();
        (void)cudaGetLastError();
        set_error("batch: could not reserve the batch arena");
        return GSI_ENOMEM;
    }
    unsigned char *pc = ctl;
    JoinArgs *d_cfg = reinterpret_cast<JoinArgs *>(pc);
    pc += sizeof(JoinArgs) * cfg.size();
    BatchQuery *d_q = reinterpret_cast<BatchQuery *>(pc);
    pc += sizeof(BatchQuery) * bqs.size();
    BatchItem *d_items = reinterpret_cast<BatchItem *>(pc);
    pc += sizeof(BatchItem) * items.size();
    BatchRec *d_recs = reinterpret_cast<BatchRec *>(pc);
    pc += sizeof(BatchRec) * items.size();
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(pc);   // [0] next item, [1] result used
    gsi_status rc = GSI_OK;
    if (cudaMemcpyAsync(d_cfg, cfg.data(), sizeof(JoinArgs) * cfg.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_q, bqs.data(), sizeof(BatchQuery) * bqs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (items.size() && cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem) * items.size(),
                                         cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaMemsetAsync(counters, 0, 16, st) != cudaSuccess) {
        set_error("batch: control upload failed");
        rc = GSI_ECUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    if (rc == GSI_OK && !items.empty()) {
        BatchArgs ba;
        ba.cfgs = d_cfg;
        ba.queries = d_q;
        ba.items = d_items;
        ba.recs = d_recs;
        ba.nitems = (int64_t)items.size();
        ba.next_item = counters;
        ba.result = result;
        ba.result_cap = result_bytes / 4;
        ba.result_used = counters + 1;
        ba.arena = arena;
        ba.slice_bytes = slice;
        ba.s_bytes = s_bytes;
        ba.t_bytes = t_bytes;
        ba.item_rows = o.item_rows > 0 ? (uint64_t)o.item_rows : 0;
        k_batch<<<grid, BNT, sm, st>>>(ba);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("batch: kernel launch failed");
            rc = GSI_ECUDA;
        }
    }
    if (stats) {
        cudaEventRecord(e1, st);
    }
    std::vector<BatchRec> recs(items.size());
    if (rc == GSI_OK) {
        if ((items.size() && cudaMemcpyAsync(recs.data(), d_recs, sizeof(BatchRec) * items.size(),
                                             cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            cudaMemcpyAsync(bqs.data(), d_q, sizeof(BatchQuery) * bqs.size(), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("batch: kernel or readback failed");
            rc = GSI_ECUDA;
        }
    }
    if (stats && e0) {
        float ms = 0;
        unsigned long long hb[2] = {0, 0};
        if (rc == GSI_OK) {
            cudaEventElapsedTime(&ms, e0, e1);
            if (cudaMemcpy(hb, dstats, 16, cudaMemcpyDeviceToHost) != cudaSuccess) hb[0] = hb[1] = 0;
        }
        stats->join_ms += ms;
        stats->join_launches += items.empty() ? 0 : 1;
        stats->kernels += items.empty() ? 0 : 1;
        stats->join_bytes += hb[0];
        stats->join_items += hb[1];
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (dstats) cudaFreeAsync(dstats, st);
    if (rc != GSI_OK) {
        if (ws) free_all_ws();
        else free_all();
        return rc;
    }
    if (ws) {
        // copy each query's rows out of the reusable staging area
        for (int i = 0; i < nq; ++i) {
            BatchPlan &p = plans[i];
            if (!p.active) continue;
            p.failed = bqs[i].status != 0;
            p.count = bqs[i].count;
        }
        for (size_t j = 0; j < items.size() && rc == GSI_OK; ++j) {
            const int qi = items[j].q;
            if (bqs[qi].status || !recs[j].rows) continue;
            const uint64_t bytes = recs[j].rows * (uint64_t)plans[qi].k * 4;
            int32_t *own = nullptr;
            if (cudaMallocAsync(&own, bytes, st) != cudaSuccess ||
                cudaMemcpyAsync(own, result + recs[j].off, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                set_error("batch: result copy failed");
                rc = GSI_ENOMEM;
                if (own) cudaFreeAsync(own, st);
                break;
            }
            gsi_result::Chunk ch{own, recs[j].rows, true};
            plans[qi].chunks.push_back(ch);
        }
        if (rc == GSI_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GSI_ECUDA;
        free_all_ws();
        return rc;
    }
    // results: chunks point into the shared result arena, which the last
    // result to be destroyed releases
    auto shared = std::make_shared<ResultArena>();
    shared->ptr = result;
    shared->device = g->device;
    shared->stream = st;
    shared->own_stream = true;
    result = nullptr;
    for (size_t j = 0; j < items.size(); ++j) {
        const int qi = items[j].q;
        if (bqs[qi].status) continue;
        if (recs[j].rows) plans[qi].chunks.push_back({shared->ptr + recs[j].off, recs[j].rows});
    }
    for (int i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        if (!p.active) continue;
        p.failed = bqs[i].status != 0;
        p.count = bqs[i].count;
        p.arena = shared;
    }
    free_all();
    return GSI_OK;
}

}  // namespace gsi

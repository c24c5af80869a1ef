// Batched execution: many queries' joins in one persistent launch.
//
// Work units come from two queues.  Seed units, listed by the host, are
// (query, range of words of the query's seed bitmap C(u_first)) pairs: a CTA
// seeds its table with the set bits of its word range and runs the query's
// join steps on those rows depth-first inside its own slice of the batch
// arena (a scratch region and two table regions used in turn), with CTA-local
// scans and survivor counters.  When a step leaves more than split_rows rows
// and steps remain, the CTA keeps the first split_rows rows and moves the
// rest, in pieces of split_rows rows, to a spill area and a spill queue; any
// CTA continues such a piece from the next step.  Idle CTAs take spill units
// before new seed units, so a query whose tables grow is spread over the GPU
// instead of running on one CTA.
//
// A unit's final rows are appended to a result arena shared by all units (one
// atomic reservation per unit) and recorded in a unit record.  A unit whose
// table does not fit its slice, or whose rows do not fit the result arena,
// marks its query failed; the host runs failed queries again on the plain
// path.  Every wait (for work, for a spill unit being published) is bounded:
// a CTA that gives up sets the error word and returns, and the host then
// treats every query of the batch as failed.
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
constexpr uint64_t SPILL_SLOTS = 1ull << 16;                  // spill queue capacity (units)
constexpr unsigned long long WAIT_SPIN_LIMIT = 1ull << 26;    // x ~100 ns sleeps: several seconds
constexpr long long UNIT_DONE = -(1ll << 62);

struct BatchQuery {
    const uint32_t *seed_bm;       // bitmap of C(u_first)
    int32_t k;
    int32_t count_only;
    unsigned status;               // 1 = failed (table or result arena overflow)
    unsigned pad;
    unsigned long long count;      // embeddings (summed over units)
};

struct BatchItem {                 // a seed unit
    int32_t q;
    int32_t pad;
    int64_t word_lo, word_hi;
};

struct SpillUnit {                 // rows of a table to continue from step t
    int32_t q;
    int32_t t;
    unsigned long long off;        // int32 offset of the rows in the spill area
    unsigned long long rows;
};

struct BatchRec {                  // one per unit that kept rows
    int32_t q;
    int32_t pad;
    unsigned long long off;        // int32 offset of the unit's rows in the result arena
    unsigned long long rows;
};

struct BatchCtl {                  // zeroed by the host, except `pending`
    unsigned long long next_item;  // seed queue head
    unsigned long long result_used;
    unsigned long long spill_used; // int32 elements
    unsigned long long sq_head, sq_tail;
    unsigned long long pending;    // units listed or queued and not yet finished
    unsigned long long nrecs;
    unsigned long long units;      // units processed (seed + spill)
    unsigned error;                // 1: a wait ran past its limit
    unsigned pad;
};

struct BatchArgs {
    const JoinArgs *cfgs;          // [q * 32 + t]
    BatchQuery *queries;
    const BatchItem *items;
    int64_t nitems;
    BatchRec *recs;
    SpillUnit *sq;
    unsigned *sq_ready;
    unsigned long long sq_cap;
    int32_t *spill;
    unsigned long long spill_cap;  // int32 elements
    BatchCtl *ctl;
    int32_t *result;               // result arena
    unsigned long long result_cap; // int32 elements
    unsigned char *arena;          // per-CTA slices
    uint64_t slice_bytes, s_bytes, t_bytes;
    uint64_t split_rows;           // 0: never split
    unsigned long long spin_limit;
};

__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Thread 0 only: the next unit (seed item >= 0, spill slot s as -(s + 1)),
// or UNIT_DONE once no unit is pending (or a wait ran out).
__device__ long long next_unit(const BatchArgs &b) {
    BatchCtl *c = b.ctl;
    unsigned long long spins = 0;
    for (;;) {
        const unsigned long long h = vload(&c->sq_head), tl = vload(&c->sq_tail);
        if (h < tl) {
            if (atomicCAS(&c->sq_head, h, h + 1) != h) continue;
            // the producer reserved slot h and is publishing it
            while (*reinterpret_cast<volatile unsigned *>(&b.sq_ready[h]) == 0u) {
                if (++spins > b.spin_limit) {
                    atomicOr(&c->error, 1u);
                    return UNIT_DONE;
                }
                __nanosleep(32);
            }
            __threadfence();
            return -(long long)h - 1;
        }
        if (vload(&c->next_item) < (unsigned long long)b.nitems) {
            const unsigned long long i = atomicAdd(&c->next_item, 1ull);
            if (i < (unsigned long long)b.nitems) return (long long)i;
        }
        if (vload(&c->pending) == 0) return UNIT_DONE;
        if (*reinterpret_cast<volatile unsigned *>(&c->error)) return UNIT_DONE;
        if (++spins > b.spin_limit) {
            atomicOr(&c->error, 1u);
            return UNIT_DONE;
        }
        __nanosleep(64);
    }
}

__global__ void __launch_bounds__(BNT) k_batch(const __grid_constant__ BatchArgs b) {
    __shared__ unsigned long long wt[BNT / 32];
    __shared__ long long unit_s;
    __shared__ unsigned long long cnt_s, off_s, slot_s;
    __shared__ int fail_s, skip_s;
    unsigned char *slice = b.arena + (uint64_t)blockIdx.x * b.slice_bytes;
    uint64_t *S = reinterpret_cast<uint64_t *>(slice);
    int32_t *reg[2] = {reinterpret_cast<int32_t *>(slice + b.s_bytes),
                       reinterpret_cast<int32_t *>(slice + b.s_bytes + b.t_bytes)};
    const uint64_t S_words = b.s_bytes / 8;
    const uint64_t W = (uint64_t)JOIN_ROW_WEIGHT;
    BatchCtl *c = b.ctl;

    for (;;) {
        if (threadIdx.x == 0) unit_s = next_unit(b);
        __syncthreads();
        const long long unit = unit_s;
        if (unit == UNIT_DONE) return;
        int q, t0, oreg;
        const int32_t *M;
        uint64_t R = 0;
        if (unit >= 0) {
            const BatchItem it = b.items[unit];
            q = it.q;
            t0 = 1;
            oreg = 1;
            M = reg[0];
        } else {
            const SpillUnit su = b.sq[-unit - 1];
            q = su.q;
            t0 = su.t;
            oreg = 0;
            M = b.spill + su.off;
            R = su.rows;
        }
        BatchQuery *bq = b.queries + q;
        const int k = bq->k;
        if (threadIdx.x == 0) skip_s = *reinterpret_cast<volatile unsigned *>(&bq->status) != 0u;
        __syncthreads();
        const bool skip = skip_s != 0;            // the query already failed: its rerun redoes this work
        if (unit >= 0 && !skip) {
            // ---- seed: set bits of the item's words, ascending
            const BatchItem it = b.items[unit];
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
            __syncthreads();                      // step 1 reads seeds written by other threads
        }
        bool failed = false;
        uint64_t cap = 0;
        for (int t = t0; t < k && R > 0 && !skip; ++t) {
            const JoinArgs &a = b.cfgs[(size_t)q * GSI_MAX_QUERY_VERTICES + t];
            int32_t *out = reg[oreg];
            if ((R + 1) * 8 + 64 > S_words * 8) { failed = true; break; }
            uint64_t *F = S;
            // bounds and slot offsets (CTA-local scan)
            unsigned long long run = 0;
            for (uint64_t base = 0; base < R; base += BNT) {
                const uint64_t i = base + threadIdx.x;
                unsigned long long v = 0;
                if (i < R) v = (unsigned long long)row_bound(a.s, M + i * (uint64_t)a.s.t, a.off, a.cl) + W;
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
                unsigned long long cn = 0;
                for (uint64_t j = threadIdx.x; j <= lim; j += BNT) cn += F[r_lo + j] <= s_next;
                cn = block_sum<BNT, unsigned long long>(cn, wt);
                const int64_t r_next = r_lo + (int64_t)cn - 1;
                join_tile<BNT, BVT>(a, M, (int64_t)R, F, total, r_lo, r_next, out, cap, &cnt_s, tile);
                r_lo = r_next;
            }
            __syncthreads();
            const uint64_t cnt = cnt_s;
            if (!last && cnt > cap) { failed = true; break; }
            M = out;
            oreg ^= 1;
            R = cnt;
            // ---- split: keep split_rows rows, queue the rest for other CTAs
            if (!last && b.split_rows && R > b.split_rows) {
                const uint64_t keep = b.split_rows, extra = R - keep;
                const uint64_t w = (uint64_t)(t + 1);
                const uint64_t nch = (extra + keep - 1) / keep;
                if (threadIdx.x == 0) {
                    off_s = ~0ull;
                    const unsigned long long sp = atomicAdd(&c->spill_used, extra * w);
                    if (sp + extra * w <= b.spill_cap) {
                        unsigned long long tl = vload(&c->sq_tail);
                        while (tl + nch <= b.sq_cap) {
                            const unsigned long long old = atomicCAS(&c->sq_tail, tl, tl + nch);
                            if (old == tl) {
                                off_s = sp;
                                slot_s = tl;
                                atomicAdd(&c->pending, (unsigned long long)nch);
                                break;
                            }
                            tl = old;
                        }
                    }
                }
                __syncthreads();
                const unsigned long long sp = off_s;
                if (sp != ~0ull) {
                    const int32_t *src = M + keep * w;
                    int32_t *dst = b.spill + sp;
                    const uint64_t n = extra * w;
                    for (uint64_t i = threadIdx.x; i < n; i += BNT) dst[i] = src[i];
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        __threadfence();
                        const unsigned long long s0 = slot_s;
                        for (uint64_t ch = 0; ch < nch; ++ch) {
                            SpillUnit u;
                            u.q = q;
                            u.t = t + 1;
                            u.off = sp + ch * keep * w;
                            u.rows = min(keep, extra - ch * keep);
                            b.sq[s0 + ch] = u;
                        }
                        __threadfence();
                        for (uint64_t ch = 0; ch < nch; ++ch) atomicExch(&b.sq_ready[s0 + ch], 1u);
                    }
                    R = keep;
                }
            }
        }
        if (!skip && k == 1) cap = bq->count_only ? 0 : b.t_bytes / 4;
        // the final table must also have fit (rows past the region are lost)
        if (!skip && !failed && !bq->count_only && R > cap) failed = true;
        // ---- final rows to the result arena
        const uint64_t rows = (skip || failed) ? 0 : min(R, cap);
        if (threadIdx.x == 0) {
            fail_s = failed;
            off_s = 0;
            if (!skip && !failed && rows > 0) {
                const unsigned long long need = rows * (unsigned long long)k;
                const unsigned long long o = atomicAdd(&c->result_used, need);
                if (o + need > b.result_cap) fail_s = 1;
                else off_s = o;
            }
            if (fail_s) atomicOr(&bq->status, 1u);
            else if (!skip) atomicAdd(&bq->count, (unsigned long long)R);
            if (!fail_s && rows > 0) {
                const unsigned long long r = atomicAdd(&c->nrecs, 1ull);
                BatchRec rec;
                rec.q = q;
                rec.pad = 0;
                rec.off = off_s;
                rec.rows = rows;
                b.recs[r] = rec;
            }
        }
        __syncthreads();
        if (!fail_s && rows > 0) {
            int32_t *dst = b.result + off_s;
            const uint64_t n = rows * (uint64_t)k;
            for (uint64_t i = threadIdx.x; i < n; i += BNT) dst[i] = __ldcg(M + i);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&c->units, 1ull);
            __threadfence();
            atomicAdd(&c->pending, ~0ull);        // this unit is finished (its children were added first)
        }
    }
}

// Copies every kept unit's rows from the staging area to its place in one
// tight buffer (dst[j] in int32 elements; ~0 = not kept), one CTA per record.
__global__ void __launch_bounds__(256) k_gather(const BatchQuery *__restrict__ queries,
                                                const BatchRec *__restrict__ recs,
                                                const unsigned long long *__restrict__ dst,
                                                const int32_t *__restrict__ src, int32_t *__restrict__ out,
                                                int64_t nrecs) {
    for (int64_t j = blockIdx.x; j < nrecs; j += gridDim.x) {
        const unsigned long long d = dst[j];
        if (d == ~0ull) continue;
        const uint64_t n = recs[j].rows * (uint64_t)queries[recs[j].q].k;
        const int32_t *s = src + recs[j].off;
        int32_t *o = out + d;
        for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) o[i] = s[i];
    }
}

}  // namespace

// Runs the planned queries of a batch in one k_batch launch; fills each
// plan's count, failed flag and row chunks.
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
        if (dstats) cudaFreeAsync(dstats, st);
        set_error("batch: shared memory need exceeds 200 KB");
        return GSI_EINVAL;
    }
    int dev = 0, nsm = 152, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    GSI_CUDA_TRY(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    GSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BNT, sm));
    if (per_sm < 1) {
        if (dstats) cudaFreeAsync(dstats, st);
        set_error("batch: kernel does not fit on an SM");
        return GSI_EINVAL;
    }
    // memory: result arena 30% and work area 70% of the budget (a workspace
    // brings its own); the work area is a quarter spill area and three
    // quarters per-CTA slices (scratch 20%, two tables 40% each), with fewer
    // CTAs when the slices would be too small
    const uint64_t align = 256, min_table = 1ull << 20;
    const uint64_t result_bytes = ws ? ws->result_bytes : (budget * 3 / 10) / align * align;
    const uint64_t work_bytes = ws ? ws->arena_bytes : (budget - result_bytes) / align * align;
    const uint64_t split_rows = o.item_rows < 0 ? 0 : (o.item_rows > 0 ? (uint64_t)o.item_rows : 4096);
    const uint64_t spill_bytes = split_rows ? (work_bytes / 4) / align * align : 0;
    const uint64_t slices_bytes = work_bytes - spill_bytes;
    int grid = nsm * per_sm;
    while (grid > 1 && (slices_bytes / (uint64_t)grid) * 2 / 5 < min_table) grid /= 2;
    const uint64_t slice = (slices_bytes / (uint64_t)grid) / align * align;
    const uint64_t s_bytes = (slice / 5) / align * align;
    const uint64_t t_bytes = ((slice - s_bytes) / 2) / align * align;
    if (t_bytes < min_table) {
        for (BatchPlan &p : plans)                        // too small for any slice: all on the plain path
            if (p.active) p.failed = true;
        if (dstats) cudaFreeAsync(dstats, st);
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
    // control block: [configs][queries][items][records][gather offsets][spill units][spill ready][ctl]
    const uint64_t sq_cap = split_rows ? SPILL_SLOTS : 0;
    const uint64_t rec_cap = items.size() + sq_cap;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t o_q = up(sizeof(JoinArgs) * cfg.size());
    const size_t o_items = o_q + up(sizeof(BatchQuery) * bqs.size());
    const size_t o_recs = o_items + up(sizeof(BatchItem) * items.size());
    const size_t o_dst = o_recs + up(sizeof(BatchRec) * rec_cap);
    const size_t o_sq = o_dst + up(sizeof(unsigned long long) * rec_cap);
    const size_t o_ready = o_sq + up(sizeof(SpillUnit) * sq_cap);
    const size_t o_ctl = o_ready + up(sizeof(unsigned) * sq_cap);
    const size_t ctl_bytes = o_ctl + up(sizeof(BatchCtl));
    unsigned char *ctl = nullptr, *arena = nullptr;
    int32_t *result = nullptr;
    auto free_all = [&]() {
        if (ctl) cudaFreeAsync(ctl, st);
        if (!ws && arena) cudaFreeAsync(arena, st);
        if (!ws && result) cudaFreeAsync(result, st);
        if (dstats) cudaFreeAsync(dstats, st);
    };
    if (ws) {
        arena = ws->arena;
        result = ws->result;
    }
    if (cudaMallocAsync(&ctl, ctl_bytes, st) != cudaSuccess ||
        (!ws && cudaMallocAsync(&arena, work_bytes, st) != cudaSuccess) ||
        (!ws && cudaMallocAsync(&result, result_bytes, st) != cudaSuccess)) {
        free_all();
        (void)cudaGetLastError();
        set_error("batch: could not reserve the batch arena");
        return GSI_ENOMEM;
    }
    JoinArgs *d_cfg = reinterpret_cast<JoinArgs *>(ctl);
    BatchQuery *d_q = reinterpret_cast<BatchQuery *>(ctl + o_q);
    BatchItem *d_items = reinterpret_cast<BatchItem *>(ctl + o_items);
    BatchRec *d_recs = reinterpret_cast<BatchRec *>(ctl + o_recs);
    unsigned long long *d_dst = reinterpret_cast<unsigned long long *>(ctl + o_dst);
    SpillUnit *d_sq = reinterpret_cast<SpillUnit *>(ctl + o_sq);
    unsigned *d_ready = reinterpret_cast<unsigned *>(ctl + o_ready);
    BatchCtl *d_ctl = reinterpret_cast<BatchCtl *>(ctl + o_ctl);
    BatchCtl hctl;
    std::memset(&hctl, 0, sizeof hctl);
    hctl.pending = items.size();
    gsi_status rc = GSI_OK;
    if (cudaMemcpyAsync(d_cfg, cfg.data(), sizeof(JoinArgs) * cfg.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_q, bqs.data(), sizeof(BatchQuery) * bqs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (items.size() && cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem) * items.size(),
                                         cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        (sq_cap && cudaMemsetAsync(d_ready, 0, sizeof(unsigned) * sq_cap, st) != cudaSuccess) ||
        cudaMemcpyAsync(d_ctl, &hctl, sizeof hctl, cudaMemcpyHostToDevice, st) != cudaSuccess) {
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
        ba.nitems = (int64_t)items.size();
        ba.recs = d_recs;
        ba.sq = d_sq;
        ba.sq_ready = d_ready;
        ba.sq_cap = sq_cap;
        ba.spill = reinterpret_cast<int32_t *>(arena + slices_bytes);
        ba.spill_cap = spill_bytes / 4;
        ba.ctl = d_ctl;
        ba.result = result;
        ba.result_cap = result_bytes / 4;
        ba.arena = arena;
        ba.slice_bytes = slice;
        ba.s_bytes = s_bytes;
        ba.t_bytes = t_bytes;
        ba.split_rows = split_rows;
        ba.spin_limit = WAIT_SPIN_LIMIT;
        k_batch<<<grid, BNT, sm, st>>>(ba);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("batch: kernel launch failed");
            rc = GSI_ECUDA;
        }
    }
    if (stats) cudaEventRecord(e1, st);
    // read back the control block, the queries and the unit records
    BatchCtl rctl;
    std::memset(&rctl, 0, sizeof rctl);
    std::vector<BatchRec> recs;
    if (rc == GSI_OK) {
        if (cudaMemcpyAsync(&rctl, d_ctl, sizeof rctl, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(bqs.data(), d_q, sizeof(BatchQuery) * bqs.size(), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("batch: kernel or readback failed");
            rc = GSI_ECUDA;
        }
    }
    if (rc == GSI_OK && rctl.nrecs) {
        recs.resize(rctl.nrecs);
        if (cudaMemcpyAsync(recs.data(), d_recs, sizeof(BatchRec) * recs.size(), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("batch: record readback failed");
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
        stats->tiles += rctl.units;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (rc != GSI_OK) {
        free_all();
        return rc;
    }
    // a wait that ran out leaves units undone: every query goes to the plain path
    const bool all_failed = rctl.error != 0;
    for (int i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        if (!p.active) continue;
        p.failed = all_failed || bqs[i].status != 0;
        p.count = bqs[i].count;
    }
    if (ws) {
        // gather every kept query's rows out of the reusable staging area into
        // one tight buffer (each query's rows contiguous), which the batch's
        // results share
        std::vector<unsigned long long> dst(recs.size(), ~0ull);
        std::vector<uint64_t> qrows((size_t)nq, 0), qoff((size_t)nq, 0);
        for (const BatchRec &r : recs)
            if (!plans[r.q].failed) qrows[r.q] += r.rows;
        uint64_t tot = 0;
        for (int i = 0; i < nq; ++i) {
            qoff[i] = tot;
            tot += qrows[i] * (uint64_t)plans[i].k;
        }
        std::vector<uint64_t> fill(qoff);
        for (size_t j = 0; j < recs.size(); ++j) {
            const BatchRec &r = recs[j];
            if (plans[r.q].failed) continue;
            dst[j] = fill[r.q];
            fill[r.q] += r.rows * (uint64_t)plans[r.q].k;
        }
        int32_t *buf = nullptr;
        if (tot > 0) {
            if (cudaMallocAsync(&buf, tot * 4, st) != cudaSuccess ||
                cudaMemcpyAsync(d_dst, dst.data(), sizeof(unsigned long long) * dst.size(), cudaMemcpyHostToDevice,
                                st) != cudaSuccess) {
                set_error("batch: result buffer or gather upload failed");
                rc = GSI_ENOMEM;
            } else {
                const int gblocks = (int)std::min<size_t>(recs.size(), (size_t)nsm * 8);
                k_gather<<<gblocks, 256, 0, st>>>(d_q, d_recs, d_dst, result, buf, (int64_t)recs.size());
                if (stats) {
                    stats->kernels += 1;
                    stats->other_launches += 1;
                }
                if (cudaGetLastError() != cudaSuccess) {
                    set_error("batch: gather launch failed");
                    rc = GSI_ECUDA;
                }
            }
        }
        if (rc == GSI_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GSI_ECUDA;
        if (rc == GSI_OK && buf) {
            auto shared = std::make_shared<ResultArena>();
            shared->ptr = buf;
            shared->device = g->device;
            shared->stream = st;
            shared->own_stream = true;
            for (int i = 0; i < nq; ++i) {
                BatchPlan &p = plans[i];
                if (!p.active || p.failed || !qrows[i]) continue;
                p.chunks.push_back({buf + qoff[i], qrows[i]});
                p.arena = shared;
            }
        } else if (buf) {
            cudaFreeAsync(buf, st);
        }
        free_all();
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
    for (const BatchRec &r : recs)
        if (!plans[r.q].failed) plans[r.q].chunks.push_back({shared->ptr + r.off, r.rows});
    for (int i = 0; i < nq; ++i)
        if (plans[i].active) plans[i].arena = shared;
    free_all();
    return GSI_OK;
}

}  // namespace gsi

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
#include "join_rows.cuh"
#include "join_tile.cuh"
#include "runtime.h"

namespace gsi {
namespace {

constexpr int BVT = JOIN_VT;
constexpr uint64_t SPILL_SLOTS = 1ull << 18;                  // spill queue capacity (units)
constexpr unsigned long long WAIT_SPIN_LIMIT = 1ull << 26;    // x ~100 ns sleeps: several seconds
constexpr long long UNIT_DONE = -(1ll << 62);

struct BatchQuery {
    const uint32_t *seed_bm;       // bitmap of C(u_first)
    int32_t k;
    int32_t count_only;
    unsigned status;               // 1 = failed (table or result arena overflow)
    int32_t cfg0;                  // the query's step t uses cfgs[cfg0 + t]
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

struct BatchCtl {                  // written by the host before every launch
    int32_t *result;               // result arena
    unsigned long long result_cap; // int32 elements
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
    const JoinArgs *cfgs;          // [cfg0 of the query + t]
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

// Drops, without a write-back, the L2 lines that lie wholly inside
// [p, p + bytes): for a CTA's own tables once they have been read for the
// last time, so that dead rows are not written to HBM when L2 evicts them.
// The contents become undefined.  Called by all threads between a barrier
// after the last read and one before the next write of the range.
template <int NT>
__device__ __forceinline__ void discard_l2(const void *p, uint64_t bytes) {
    const uint64_t a = (uint64_t)reinterpret_cast<uintptr_t>(p);
    const uint64_t end = (a + bytes) & ~127ull;
    for (uint64_t x = ((a + 127) & ~127ull) + 128ull * threadIdx.x; x < end; x += 128ull * NT)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(x) : "memory");
}

// One instance per block shape: NT threads per CTA, RPT rows per thread in
// the row pass (the batched autotuner picks one).
template <int NT, int RPT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_batch(const __grid_constant__ BatchArgs b) {
    constexpr int BNT = NT, BNV = NT * BVT;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long wt[BNT / 32];
    __shared__ long long unit_s;
    __shared__ unsigned long long cnt_s, lcnt_s, off_s, slot_s;
    __shared__ unsigned rfail_s;
    __shared__ int fail_s, skip_s;
    __shared__ __align__(16) JoinArgs a_s;
    unsigned char *slice = b.arena + (uint64_t)blockIdx.x * b.slice_bytes;
    uint64_t *S = reinterpret_cast<uint64_t *>(slice);
    int32_t *reg[2] = {reinterpret_cast<int32_t *>(slice + b.s_bytes),
                       reinterpret_cast<int32_t *>(slice + b.s_bytes + b.t_bytes)};
    const uint64_t S_words = b.s_bytes / 8;
    const uint64_t W = (uint64_t)JOIN_ROW_WEIGHT;
    BatchCtl *c = b.ctl;
    int32_t *const result = c->result;
    const unsigned long long result_cap = c->result_cap;

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
            __syncthreads();                      // the previous step's readers of a_s are done
            {   // this step's configuration in shared memory
                const uint32_t *src = reinterpret_cast<const uint32_t *>(b.cfgs + bq->cfg0 + t);
                uint32_t *dst = reinterpret_cast<uint32_t *>(&a_s);
                for (int i = threadIdx.x; i < (int)(sizeof(JoinArgs) / 4); i += BNT) dst[i] = src[i];
            }
            const JoinArgs &a = a_s;
            int32_t *out = reg[oreg];
            const bool last = t == k - 1;
            cap = b.t_bytes / (4ull * (uint64_t)(t + 1));
            if (last && bq->count_only) cap = 0;
            // long rows (bound above SHORT_MAX) and their slot offsets in the scratch region
            const LongLayout ll = long_layout(S_words, t);
            LongTable lt;
            lt.rows = reinterpret_cast<int32_t *>(S);
            lt.bnd = reinterpret_cast<uint32_t *>(lt.rows + ll.cap * (uint64_t)t);
            lt.blo = lt.bnd + ll.cap;
            lt.cap = ll.cap;
            lt.count = &lcnt_s;
            uint64_t *F = S + ll.f_off;
            if (threadIdx.x == 0) {
                cnt_s = 0;
                lcnt_s = 0;
                rfail_s = 0;
            }
            __syncthreads();
            // short rows joined inline, long rows set aside
            unsigned long long abytes = 0, items = 0, lbytes = 0;
            row_pass<BNT, true, RPT, false>(a, M, R, 0, (uint64_t)BNT * RPT, out, cap, &cnt_s, lt, &rfail_s, smem,
                                            &abytes, &items, &lbytes);
            if (a.stats) {                       // one add per step of a unit
                abytes = block_sum<BNT, unsigned long long>(abytes, wt);
                items = block_sum<BNT, unsigned long long>(items, wt);
                lbytes = block_sum<BNT, unsigned long long>(lbytes, wt);
                if (threadIdx.x == 0) {
                    if (abytes) atomicAdd(a.stats, abytes);
                    if (items) atomicAdd(a.stats + 1, items);
                    if (lbytes) atomicAdd(a.stats + 2, lbytes);
                }
            }
            __syncthreads();
            if (rfail_s) { failed = true; break; }     // long-row table full: the plain path
            const uint64_t L = lcnt_s;
            if (L > 0) {
                // the long rows through the candidate-slot tiles, CTA-local
                unsigned long long run = 0;
                for (uint64_t base = 0; base < L; base += BNT) {
                    const uint64_t i = base + threadIdx.x;
                    const unsigned long long v =
                        i < L ? (unsigned long long)(lt.bnd[i] & BOUND_LEN_MASK) + W : 0ull;
                    unsigned long long tot;
                    const unsigned long long ex = block_exclusive_scan<BNT, unsigned long long>(v, wt, &tot) + run;
                    if (i < L) F[i] = ex;
                    run += tot;
                }
                const uint64_t total = run;
                if (threadIdx.x == 0) F[L] = total;
                __syncthreads();
                // tiles in order; each tile spans at most BNV/W + 1 rows past its first
                const uint64_t ntiles = (total + BNV - 1) / BNV;
                int64_t r_lo = 0;
                const uint64_t span = BNV / W + 1;
                for (uint64_t tile = 0; tile < ntiles; ++tile) {
                    const uint64_t s_next = min((tile + 1) * (uint64_t)BNV, total);
                    const uint64_t lim = min(L - (uint64_t)r_lo, span);
                    unsigned long long cn = 0;
                    for (uint64_t j = threadIdx.x; j <= lim; j += BNT) cn += F[r_lo + j] <= s_next;
                    cn = block_sum<BNT, unsigned long long>(cn, wt);
                    const int64_t r_next = r_lo + (int64_t)cn - 1;
                    join_tile<BNT, BVT, false, true>(a, lt.rows, (int64_t)L, F, total, r_lo, r_next, out, cap, &cnt_s,
                                                     tile, lt.bnd, lt.blo);
                    r_lo = r_next;
                }
            }
            __syncthreads();
            discard_l2<BNT>(M, R * (uint64_t)t * 4);    // this step's input is dead
            const uint64_t cnt = cnt_s;
            if (a.stats && threadIdx.x == 0) {   // survivors written (both models)
                atomicAdd(a.stats, 4ull * (uint64_t)(t + 1) * min(cnt, cap));
                atomicAdd(a.stats + 2, 4ull * (uint64_t)(t + 1) * min(cnt, cap));
            }
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
                    discard_l2<BNT>(src, n * 4);       // the queued rows now live in the spill area
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
                if (o + need > result_cap) fail_s = 1;
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
            int32_t *dst = result + off_s;
            const uint64_t n = rows * (uint64_t)k;
            for (uint64_t i = threadIdx.x; i < n; i += BNT) dst[i] = __ldcg(M + i);
        }
        __syncthreads();
        if (!fail_s && rows > 0) discard_l2<BNT>(M, rows * (uint64_t)k * 4);   // copied out
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


// The batch kernel for a block shape (threads per CTA, rows per thread).
using BatchKernel = void (*)(BatchArgs);
BatchKernel batch_kernel(int nt, int rpt) {
    if (nt == 128) return rpt == 1 ? k_batch<128, 1> : k_batch<128, 2>;
    return rpt == 1 ? k_batch<256, 1> : k_batch<256, 2>;
}

// ------------------------------------------------------------------- host
// Sizes the launch, lists the seed units, builds the per-step configurations
// and reserves the control block (and the work area unless a workspace brings
// one).  With keep_template the initial query records also stay on the device
// so that replays can reset them with a device copy.
gsi_status batch_setup(BatchLaunch &L, gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &o,
                       uint64_t budget, cudaStream_t st, BatchWorkspace *ws, bool stats, bool keep_template) {
    L = BatchLaunch();
    const int nq = (int)plans.size();
    L.nq = (size_t)nq;
    if ((o.block_threads != 0 && o.block_threads != 128 && o.block_threads != 256) ||
        (o.rows_per_thread != 0 && o.rows_per_thread != 1 && o.rows_per_thread != 2) || o.isect < 0 ||
        o.isect > ISECT_BITMAP) {
        set_error("batch: block_threads must be 128 or 256, rows_per_thread 1 or 2, isect a GSI_ISECT_* value");
        return GSI_EINVAL;
    }
    L.nt = o.block_threads ? o.block_threads : 256;
    L.rpt = o.rows_per_thread ? o.rows_per_thread : 2;
    if (stats) {
        GSI_CUDA_TRY(cudaMallocAsync(&L.dstats, 24, st));
    }
    size_t sm = join_smem(LONG_RMAX, 1, 1);
    for (int i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        if (!p.active) continue;
        for (int t = 1; t < p.k; ++t) {
            sm = std::max(sm, join_smem(LONG_RMAX, p.steps[t].t, p.steps[t].d));
            sm = std::max(sm, rows_smem(L.nt, p.steps[t].t, L.rpt));
        }
    }
    if (sm > 200 * 1024) {
        set_error("batch: shared memory need exceeds 200 KB");
        return GSI_EINVAL;
    }
    L.sm = sm;
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&L.nsm, cudaDevAttrMultiProcessorCount, dev);
    const BatchKernel kern = batch_kernel(L.nt, L.rpt);
    GSI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    GSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.nt, sm));
    if (per_sm < 1) {
        set_error("batch: kernel does not fit on an SM");
        return GSI_EINVAL;
    }
    // memory: result arena 30% and work area 70% of the budget (a workspace
    // brings its own); the work area is a quarter spill area and three
    // quarters per-CTA slices (scratch 20%, two tables 40% each), with fewer
    // CTAs when the slices would be too small
    const uint64_t align = 256, min_table = 1ull << 20;
    L.result_bytes = ws ? ws->result_bytes : (budget * 3 / 10) / align * align;
    L.work_bytes = ws ? ws->arena_bytes : (budget - L.result_bytes) / align * align;
    L.split_rows = o.item_rows < 0 ? 0 : (o.item_rows > 0 ? (uint64_t)o.item_rows : 1024);
    L.spill_bytes = L.split_rows ? (L.work_bytes / 4) / align * align : 0;
    L.slices_bytes = L.work_bytes - L.spill_bytes;
    int grid = L.nsm * per_sm;
    while (grid > 1 && (L.slices_bytes / (uint64_t)grid) * 2 / 5 < min_table) grid /= 2;
    L.grid = grid;
    L.slice = (L.slices_bytes / (uint64_t)grid) / align * align;
    L.s_bytes = (L.slice / 5) / align * align;
    L.t_bytes = ((L.slice - L.s_bytes) / 2) / align * align;
    if (L.t_bytes < min_table) {
        L.all_plain = true;                 // too small for any slice: all on the plain path
        return GSI_OK;
    }
    // per-query records, step configurations and seed units
    std::vector<BatchQuery> bqs((size_t)nq);
    std::vector<JoinArgs> cfg;
    std::vector<BatchItem> items;
    const uint64_t max_words = std::max<uint64_t>(1, (L.t_bytes - 1024) / 128);   // seeds fit a table region
    for (int i = 0; i < nq; ++i) {
        BatchPlan &p = plans[i];
        std::memset(&bqs[i], 0, sizeof(BatchQuery));
        bqs[i].k = p.k;
        bqs[i].count_only = o.count_only;
        if (!p.active) continue;
        bqs[i].seed_bm = p.bitmaps + (uint64_t)p.order[0] * (uint64_t)g->nwords;
        bqs[i].cfg0 = (int32_t)cfg.size();
        cfg.resize(cfg.size() + (size_t)p.k);
        for (int t = 1; t < p.k; ++t) {
            const int co = (t == p.k - 1) && o.count_only;
            cfg[(size_t)bqs[i].cfg0 + t] =
                make_join_args(g, p.steps[t], p.bitmaps + (uint64_t)p.order[t] * (uint64_t)g->nwords, co, L.dstats);
            cfg[(size_t)bqs[i].cfg0 + t].isect = o.isect;
            cfg[(size_t)bqs[i].cfg0 + t].rmax = LONG_RMAX;     // its tiles see long rows only
        }
        // word ranges of the seed bitmap holding about seeds_per_item seeds each
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
    if (cfg.empty()) cfg.resize(1);
    L.nitems = items.size();
    L.ncfg = cfg.size();
    // control block: [configs][queries][query template][items][records][gather offsets][spill units][ready][ctl]
    L.sq_cap = L.split_rows ? SPILL_SLOTS : 0;
    L.rec_cap = items.size() + L.sq_cap;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    L.o_q = up(sizeof(JoinArgs) * cfg.size());
    L.o_tpl = L.o_q + up(sizeof(BatchQuery) * bqs.size());
    L.o_items = L.o_tpl + (keep_template ? up(sizeof(BatchQuery) * bqs.size()) : 0);
    L.o_recs = L.o_items + up(sizeof(BatchItem) * items.size());
    L.o_dst = L.o_recs + up(sizeof(BatchRec) * L.rec_cap);
    L.o_sq = L.o_dst + up(sizeof(unsigned long long) * L.rec_cap);
    L.o_ready = L.o_sq + up(sizeof(SpillUnit) * L.sq_cap);
    L.o_ctl = L.o_ready + up(sizeof(unsigned) * L.sq_cap);
    L.ctl_bytes = L.o_ctl + up(sizeof(BatchCtl));
    L.has_template = keep_template;
    if (cudaMallocAsync(&L.ctl, L.ctl_bytes, st) != cudaSuccess) {
        (void)cudaGetLastError();
        L.ctl = nullptr;
        set_error("batch: could not reserve the control block");
        return GSI_ENOMEM;
    }
    if (ws) {
        L.arena = ws->arena;
    } else {
        if (cudaMallocAsync(&L.arena, L.work_bytes, st) != cudaSuccess) {
            (void)cudaGetLastError();
            L.arena = nullptr;
            set_error("batch: could not reserve the batch arena");
            return GSI_ENOMEM;
        }
        L.own_arena = true;
    }
    GSI_CUDA_TRY(cudaMemcpyAsync(L.ctl, cfg.data(), sizeof(JoinArgs) * cfg.size(), cudaMemcpyHostToDevice, st));
    if (items.size())
        GSI_CUDA_TRY(cudaMemcpyAsync(L.ctl + L.o_items, items.data(), sizeof(BatchItem) * items.size(),
                                     cudaMemcpyHostToDevice, st));
    if (keep_template)
        GSI_CUDA_TRY(cudaMemcpyAsync(L.ctl + L.o_tpl, bqs.data(), sizeof(BatchQuery) * bqs.size(),
                                     cudaMemcpyHostToDevice, st));
    L.q_init.assign(reinterpret_cast<const unsigned char *>(bqs.data()),
                    reinterpret_cast<const unsigned char *>(bqs.data()) + sizeof(BatchQuery) * bqs.size());
    return GSI_OK;
}

// The launch's control words: counters zeroed, every seed unit pending, the
// result arena (host to device, ahead of the kernel on the stream).
gsi_status batch_enqueue_ctl(BatchLaunch &L, int32_t *result, uint64_t result_bytes, cudaStream_t st) {
    if (L.all_plain) return GSI_OK;
    BatchCtl h;
    std::memset(&h, 0, sizeof h);
    h.result = result;
    h.result_cap = result_bytes / 4;
    h.pending = L.nitems;
    GSI_CUDA_TRY(cudaMemcpyAsync(L.ctl + L.o_ctl, &h, sizeof h, cudaMemcpyHostToDevice, st));
    return GSI_OK;
}

// Query records reset, spill queue cleared, counters zeroed, then the kernel.
// With a template every step is device work only, so it can be captured.
gsi_status batch_enqueue_kernel(BatchLaunch &L, cudaStream_t st) {
    if (L.all_plain) return GSI_OK;
    BatchQuery *d_q = reinterpret_cast<BatchQuery *>(L.ctl + L.o_q);
    if (L.has_template)
        GSI_CUDA_TRY(cudaMemcpyAsync(d_q, L.ctl + L.o_tpl, L.q_init.size(), cudaMemcpyDeviceToDevice, st));
    else
        GSI_CUDA_TRY(cudaMemcpyAsync(d_q, L.q_init.data(), L.q_init.size(), cudaMemcpyHostToDevice, st));
    if (L.sq_cap) GSI_CUDA_TRY(cudaMemsetAsync(L.ctl + L.o_ready, 0, sizeof(unsigned) * L.sq_cap, st));
    if (L.dstats) GSI_CUDA_TRY(cudaMemsetAsync(L.dstats, 0, 24, st));
    if (L.nitems == 0) return GSI_OK;
    BatchArgs ba;
    ba.cfgs = reinterpret_cast<const JoinArgs *>(L.ctl);
    ba.queries = d_q;
    ba.items = reinterpret_cast<const BatchItem *>(L.ctl + L.o_items);
    ba.nitems = (int64_t)L.nitems;
    ba.recs = reinterpret_cast<BatchRec *>(L.ctl + L.o_recs);
    ba.sq = reinterpret_cast<SpillUnit *>(L.ctl + L.o_sq);
    ba.sq_ready = reinterpret_cast<unsigned *>(L.ctl + L.o_ready);
    ba.sq_cap = L.sq_cap;
    ba.spill = reinterpret_cast<int32_t *>(L.arena + L.slices_bytes);
    ba.spill_cap = L.spill_bytes / 4;
    ba.ctl = reinterpret_cast<BatchCtl *>(L.ctl + L.o_ctl);
    ba.arena = L.arena;
    ba.slice_bytes = L.slice;
    ba.s_bytes = L.s_bytes;
    ba.t_bytes = L.t_bytes;
    ba.split_rows = L.split_rows;
    ba.spin_limit = WAIT_SPIN_LIMIT;
    batch_kernel(L.nt, L.rpt)<<<L.grid, L.nt, L.sm, st>>>(ba);
    GSI_CUDA_TRY(cudaGetLastError());
    return GSI_OK;
}

// After the kernel: each plan's count, failed flag and row chunks.  With a
// workspace the kept rows are gathered into one tight buffer; otherwise the
// chunks point into `result`, which `arena` (when given) keeps alive.
gsi_status batch_collect(BatchLaunch &L, gsi_graph *g, std::vector<BatchPlan> &plans, int32_t *result,
                         std::shared_ptr<ResultArena> arena, cudaStream_t st, gsi_stats *stats, BatchWorkspace *ws) {
    const int nq = (int)plans.size();
    for (BatchPlan &p : plans) {
        p.failed = false;
        p.count = 0;
        p.chunks.clear();
        p.arena.reset();
    }
    if (L.all_plain) {
        for (BatchPlan &p : plans)
            if (p.active) p.failed = true;
        return GSI_OK;
    }
    BatchCtl rctl;
    std::memset(&rctl, 0, sizeof rctl);
    std::vector<BatchQuery> bqs((size_t)nq);
    std::vector<BatchRec> recs;
    BatchQuery *d_q = reinterpret_cast<BatchQuery *>(L.ctl + L.o_q);
    if (cudaMemcpyAsync(&rctl, L.ctl + L.o_ctl, sizeof rctl, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(bqs.data(), d_q, sizeof(BatchQuery) * bqs.size(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("batch: kernel or readback failed");
        return GSI_ECUDA;
    }
    if (rctl.nrecs) {
        recs.resize(rctl.nrecs);
        if (cudaMemcpyAsync(recs.data(), L.ctl + L.o_recs, sizeof(BatchRec) * recs.size(), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("batch: record readback failed");
            return GSI_ECUDA;
        }
    }
    if (stats) {
        unsigned long long hb[3] = {0, 0, 0};
        if (L.dstats && cudaMemcpy(hb, L.dstats, 24, cudaMemcpyDeviceToHost) != cudaSuccess) hb[0] = hb[1] = hb[2] = 0;
        stats->join_bytes += hb[0];
        stats->batch_bytes += hb[0];
        stats->join_items += hb[1];
        stats->join_bytes_listwise += hb[2];
        stats->tiles += rctl.units;
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
        gsi_status rc = GSI_OK;
        if (tot > 0) {
            unsigned long long *d_dst = reinterpret_cast<unsigned long long *>(L.ctl + L.o_dst);
            if (cudaMallocAsync(&buf, tot * 4, st) != cudaSuccess ||
                cudaMemcpyAsync(d_dst, dst.data(), sizeof(unsigned long long) * dst.size(), cudaMemcpyHostToDevice,
                                st) != cudaSuccess) {
                (void)cudaGetLastError();
                set_error("batch: result buffer or gather upload failed");
                rc = GSI_ENOMEM;
            } else {
                const int gblocks = (int)std::min<size_t>(recs.size(), (size_t)L.nsm * 8);
                k_gather<<<gblocks, 256, 0, st>>>(d_q, reinterpret_cast<const BatchRec *>(L.ctl + L.o_recs), d_dst,
                                                  result, buf, (int64_t)recs.size());
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
        return rc;
    }
    for (const BatchRec &r : recs)
        if (!plans[r.q].failed) plans[r.q].chunks.push_back({result + r.off, r.rows});
    for (int i = 0; i < nq; ++i)
        if (plans[i].active) plans[i].arena = arena;
    return GSI_OK;
}

void batch_release(BatchLaunch &L, cudaStream_t st) {
    if (L.ctl) cudaFreeAsync(L.ctl, st);
    if (L.own_arena && L.arena) cudaFreeAsync(L.arena, st);
    if (L.dstats) cudaFreeAsync(L.dstats, st);
    L = BatchLaunch();
}

// One batch launch end to end: setup, control words, kernel, collection.
gsi_status batch_run_device(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &o,
                            uint64_t budget, cudaStream_t st, gsi_stats *stats, BatchWorkspace *ws) {
    if (plans.empty()) return GSI_OK;
    BatchLaunch L;
    gsi_status rc = batch_setup(L, g, plans, o, budget, st, ws, stats != nullptr, false);
    int32_t *result = nullptr;
    std::shared_ptr<ResultArena> arena;
    if (rc == GSI_OK && !L.all_plain) {
        if (ws) {
            result = ws->result;
        } else if (cudaMallocAsync(&result, L.result_bytes, st) != cudaSuccess) {
            (void)cudaGetLastError();
            result = nullptr;
            set_error("batch: could not reserve the result arena");
            rc = GSI_ENOMEM;
        } else {
            arena = std::make_shared<ResultArena>();     // the last result to go releases it
            arena->ptr = result;
            arena->device = g->device;
            arena->stream = st;
            arena->own_stream = true;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == GSI_OK && stats && !L.all_plain) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    if (rc == GSI_OK) rc = batch_enqueue_ctl(L, result, L.result_bytes, st);
    if (rc == GSI_OK && e0) cudaEventRecord(e0, st);
    if (rc == GSI_OK) rc = batch_enqueue_kernel(L, st);
    if (rc == GSI_OK && e1) cudaEventRecord(e1, st);
    if (rc == GSI_OK) rc = batch_collect(L, g, plans, result, arena, st, stats, ws);
    if (e0) {
        float ms = 0;
        if (rc == GSI_OK) cudaEventElapsedTime(&ms, e0, e1);
        stats->join_ms += ms;
        stats->batch_ms += ms;
        stats->join_launches += L.nitems ? 1 : 0;
        stats->kernels += L.nitems ? 1 : 0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    batch_release(L, st);
    return rc;
}

}  // namespace gsi

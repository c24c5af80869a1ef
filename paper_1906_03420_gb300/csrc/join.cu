// Join iterations (Sec. V, Algs. 3-4), in two forms.
//
// Host-sized (gsi_join_step, and the splitting path of the memory-bounded
// driver): one iteration as three launches,
//   1. scan   F[i] = sum_{r<i} (cap_r + W), where cap_r bounds row r's output
//             (Alg. 4's preallocation bound), plus W "row slots" per row that
//             pay for staging the row (load balancing, below);
//   2. part   for every tile of NV consecutive slots, its first row;
//   3. join   the fused kernel: one CTA per tile of NV slots.
//
// Device-driven (k_query): the seed and every iteration of one query in one
// cooperative launch, the same three phases separated by bounded grid
// barriers, tiles taken from a counter.  Its bound scan also keeps each row's
// shortest sub-list (start, length, linking edge), so the join tiles stage
// rows without searching again.
//
// Output bound.  Every neighbour list N(v,l) is stored sorted by (label rank
// of the neighbour, neighbour id), so the neighbours of v via l that carry
// the new query vertex's label form one contiguous, id-sorted sub-list.  Any
// survivor w of row i lies in that sub-list of every linking edge, so each
// row takes as its candidate list (and output bound, Alg. 4) the shortest of
// these sub-lists; Alg. 4's global choice of the least frequent edge label is
// the same bound taken once for all rows.
//
// Work decomposition.  Instead of the paper's warp-per-row with a 4-layer
// balance scheme and dynamically launched child kernels (Sec. VI-A), every
// candidate of every row is one slot of a flat index space whose row offsets
// are F, and each CTA takes a fixed NV slots.  A hub row with 10^5
// candidates is spread over many CTAs; rows with one candidate are packed
// NV/W to a CTA.  The W per-row slots bound the rows one CTA stages, so its
// shared memory holds every row it touches.
//
// Per CTA (Sec. V "GPU-friendly set operation"):
//   * the partial matches m_i of its rows are staged in shared memory with
//     the bounds of every label sub-list they need (small lists);
//   * a slot -> row map is built with one block-wide max-scan;
//   * slots read consecutive elements of the row's candidate sub-list
//     (coalesced medium list);
//   * C(u) is probed as a bitset, one 4-byte load per candidate (large list);
//   * set subtraction (w not in m_i) is checked against the staged row;
//   * the other linking edges test w in their sub-list by binary search (the
//     intersection), only for candidates that survived the cheaper checks;
//   * survivors are compacted with one block-wide prefix sum and one global
//     atomic per CTA, then written once as rows of M' (Prealloc-Combine: the
//     join runs once; the output buffer is sized by F's total).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"
#include "join_rows.cuh"
#include "join_tile.cuh"
#include "scan.cuh"

namespace gsi {
namespace {

// Reduce pass: stores each row's bound for the down pass.
struct CapStoreProducer {
    const int32_t *M;
    const uint32_t *off;
    const uint16_t *cl;
    uint32_t *caps;
    uint64_t W;
    StepDev s;
    __device__ uint64_t operator()(int64_t i) const {
        uint32_t c = row_bound(s, M + i * s.t, off, cl);
        caps[i] = c;
        return (uint64_t)c + W;
    }
};
struct CapLoadProducer {
    const uint32_t *caps;
    uint64_t W;
    __device__ uint64_t operator()(int64_t i) const { return (uint64_t)caps[i] + W; }
};


template <typename P1, typename P2, typename Wr>
cudaError_t two_producer_scan(P1 p1, P2 p2, int64_t n, Wr write, uint64_t *scratch, cudaStream_t st) {
    if (n <= 0) {
        k_scan_empty<uint64_t, Wr><<<1, 1, 0, st>>>(write);
        return cudaGetLastError();
    }
    int64_t nb = scan_blocks(n);
    k_scan_reduce<uint64_t, P1><<<(unsigned)nb, SCAN_NT, 0, st>>>(p1, n, scratch);
    k_scan_spine<uint64_t><<<1, 1024, 0, st>>>(scratch, nb);
    k_scan_down<uint64_t, P2, Wr><<<(unsigned)nb, SCAN_NT, 0, st>>>(p2, n, scratch, nb, write);
    return cudaGetLastError();
}

__global__ void k_partition(const uint64_t *__restrict__ F, int64_t R, uint64_t total, int64_t ntiles,
                            int64_t *__restrict__ part) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > ntiles) return;
    uint64_t s = (uint64_t)b * JOIN_NV;
    if (s > total) s = total;
    int64_t lo = 0, hi = R;            // largest r in [0, R] with F[r] <= s
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (F[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    part[b] = lo;
}

template <int NT, int VT>
__global__ void __launch_bounds__(NT) k_join(const __grid_constant__ JoinArgs a) {
    join_tile<NT, VT>(a, a.M, a.R, a.F, a.total, a.part[blockIdx.x], a.part[blockIdx.x + 1], a.out, a.out_cap,
                      a.out_count, blockIdx.x);
}

// ------------------------------------------------- one launch per query
// The whole join of one query in a single cooperative launch: the seed, then
// for every step the bound scan, the tile partition and the join tiles, with
// a grid barrier between phases.  All CTAs are co-resident (cooperative
// launch), so the barrier is a counter and a generation word; every wait is
// bounded, and a CTA that gives up sets an error bit and returns, as does
// every CTA that later sees the bit, so the kernel always terminates.

constexpr unsigned long long BARRIER_SPIN_LIMIT = 1ull << 24;   // x ~64 ns sleeps: about a second

__device__ __forceinline__ bool grid_barrier(QueryCtl *ctl, unsigned nblocks) {
    const unsigned long long limit = ctl->spin_limit ? ctl->spin_limit : BARRIER_SPIN_LIMIT;
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &ctl->bar_gen;
        volatile unsigned *fail = &ctl->fail;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*gen == g) {
                if (*fail & 4u) { ok = 0; break; }
                if (++spins > limit) {
                    atomicOr(&ctl->fail, 4u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok && !(*fail & 4u);
    }
    __syncthreads();
    return ok_s != 0;
}

// Sum of v over this CTA's predecessors (j < blockIdx.x) and over all CTAs.
__device__ __forceinline__ void cta_prefix(const unsigned long long *bsum, unsigned nblocks, unsigned long long *wt,
                                           unsigned long long *pre, unsigned long long *tot) {
    unsigned long long p = 0, q = 0;
    for (unsigned j = threadIdx.x; j < nblocks; j += blockDim.x) {
        const unsigned long long v = __ldcg(bsum + j);
        q += v;
        if (j < blockIdx.x) p += v;
    }
    *pre = block_sum<JOIN_NT, unsigned long long>(p, wt);
    *tot = block_sum<JOIN_NT, unsigned long long>(q, wt);
}

// The long rows of a step (bound above SHORT_MAX) through the candidate-slot
// tiles: per-CTA slot sums, slot offsets F, the first row of every tile, then
// the tiles dealt round-robin over the CTAs, with a grid barrier after each
// phase.  Survivors
// join those of the row pass in st->out.  False when a barrier wait gave up
// or the partition does not fit (fail bit 1).
template <int NT, int VT>
__device__ __forceinline__ bool long_rows_join(const JoinArgs &a, DStep *st, QueryCtl *ctl, const LongTable &lt,
                                               uint64_t L, uint64_t *F, int64_t *part, uint64_t part_cap,
                                               uint64_t cap, unsigned long long *bsum, unsigned long long *wt) {
    constexpr int NV = NT * VT;
    const unsigned G = gridDim.x;
    const uint64_t W = (uint64_t)JOIN_ROW_WEIGHT;
    unsigned long long pre, tot;
    // slots of each long row: its bound plus W staging slots; per-CTA sums
    const uint64_t per = (L + G - 1) / G;
    const uint64_t chunk = (per + SCAN_NV - 1) / SCAN_NV * SCAN_NV;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = min(L, lo + chunk);
    unsigned long long sum = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += NT) sum += (unsigned long long)(__ldcg(lt.bnd + i) & BOUND_LEN_MASK) + W;
    sum = block_sum<NT, unsigned long long>(sum, wt);
    if (threadIdx.x == 0) bsum[blockIdx.x] = sum;
    if (!grid_barrier(ctl, G)) return false;
    // slot offsets F over the long rows
    cta_prefix(bsum, G, wt, &pre, &tot);
    const uint64_t total = tot;
    const uint64_t ntiles = (total + NV - 1) / NV;
    if (ntiles + 1 > part_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->fail, 1u);
        return false;
    }
    {
        unsigned long long run = pre;
        for (uint64_t base = lo; base < hi; base += NT) {
            const uint64_t i = base + threadIdx.x;
            const unsigned long long v = i < hi ? (unsigned long long)(__ldcg(lt.bnd + i) & BOUND_LEN_MASK) + W : 0ull;
            unsigned long long t2;
            const unsigned long long ex = block_exclusive_scan<NT, unsigned long long>(v, wt, &t2) + run;
            if (i < hi) F[i] = ex;
            run += t2;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        F[L] = total;
        st->total = total;
        st->ntiles = ntiles;
    }
    if (!grid_barrier(ctl, G)) return false;
    // first long row of every tile
    for (uint64_t b = (uint64_t)blockIdx.x * NT + threadIdx.x; b <= ntiles; b += (uint64_t)G * NT) {
        const uint64_t sl = min(b * (uint64_t)NV, total);
        int64_t l2 = 0, h2 = (int64_t)L;
        while (l2 < h2) {
            int64_t mid = (l2 + h2 + 1) >> 1;
            if (__ldcg(F + mid) <= sl) l2 = mid;
            else h2 = mid - 1;
        }
        part[b] = l2;
    }
    if (!grid_barrier(ctl, G)) return false;
    // the join tiles, dealt round-robin: every tile holds the same number of
    // candidate slots, so no counter is needed to balance them
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += G) {
        __syncthreads();                  // the previous tile's readers of shared memory are done
        join_tile<NT, VT, false, true>(a, lt.rows, (int64_t)L, F, total, __ldcg(part + tile), __ldcg(part + tile + 1),
                                       st->out, cap, &st->count, tile, lt.bnd, lt.blo);
    }
    return grid_barrier(ctl, G);
}

template <int NT, int VT, bool LW>
__global__ void __launch_bounds__(NT, 4) k_query(const JoinArgs *__restrict__ cfgs, DStep *steps, int k, QueryCtl *ctl,
                                              const uint32_t *__restrict__ seed_bitmap, int64_t nwords,
                                              unsigned long long *bsum) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long wt[NT / 32];
    __shared__ __align__(16) JoinArgs a_s;
    const unsigned G = gridDim.x;
    unsigned long long pre, tot;

    // ---- seed: C(u_first) as the one-column table in the first region (Alg. 2)
    int32_t *seed_out = const_cast<int32_t *>(steps[1].M);
    {
        const uint64_t per = ((uint64_t)nwords + G - 1) / G;
        const uint64_t chunk = (per + SCAN_NV - 1) / SCAN_NV * SCAN_NV;
        const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = min((uint64_t)nwords, lo + chunk);
        unsigned long long c = 0;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += NT) c += __popc(seed_bitmap[i]);
        c = block_sum<NT, unsigned long long>(c, wt);
        if (threadIdx.x == 0) bsum[blockIdx.x] = c;
        if (!grid_barrier(ctl, G)) return;
        cta_prefix(bsum, G, wt, &pre, &tot);
        unsigned long long run = pre;
        for (uint64_t base = lo; base < hi; base += NT) {
            const uint64_t i = base + threadIdx.x;
            const uint32_t b = i < hi ? seed_bitmap[i] : 0u;
            unsigned long long t2;
            unsigned long long pos = block_exclusive_scan<NT, unsigned long long>(__popc(b), wt, &t2) + run;
            uint32_t x = b;
            while (x) {
                seed_out[pos++] = (int32_t)(i * 32 + (uint64_t)(__ffs(x) - 1));
                x &= x - 1;
            }
            run += t2;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) steps[0].count = tot;
        if (!grid_barrier(ctl, G)) return;
    }

    for (int t = 1; t < k; ++t) {
        DStep *st = steps + t;
        {   // this step's configuration, once per CTA, in shared memory
            const uint32_t *src = reinterpret_cast<const uint32_t *>(cfgs + t);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&a_s);
            for (int i = threadIdx.x; i < (int)(sizeof(JoinArgs) / 4); i += NT) dst[i] = src[i];
        }
        const JoinArgs &a = a_s;
        const uint64_t R = __ldcg(&steps[t - 1].count);
        // the previous table must have fit its region
        if (t > 1 && R > __ldcg(&steps[t - 1].out_cap)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->fail, 2u);
            return;
        }
        const LongLayout ll = long_layout(st->S_words, t);
        LongTable lt;
        lt.rows = reinterpret_cast<int32_t *>(st->S);
        lt.bnd = reinterpret_cast<uint32_t *>(lt.rows + ll.cap * (uint64_t)t);
        lt.blo = lt.bnd + ll.cap;
        lt.cap = ll.cap;
        lt.count = &st->nlong;
        uint64_t cap = st->out_bytes / (4ull * (uint64_t)(t + 1));
        if (st->row_cap && st->row_cap < cap) cap = st->row_cap;
        if (st->count_only) cap = 0;
        if (blockIdx.x == 0 && threadIdx.x == 0) st->out_cap = cap;
        __syncthreads();
        // ---- short rows joined inline, long rows set aside (one pass over M)
        unsigned long long abytes = 0, items = 0, lbytes = 0;
        row_pass<NT, true, ROW_RPT, LW>(a, st->M, R, (uint64_t)blockIdx.x * NT * ROW_RPT, (uint64_t)G * NT * ROW_RPT,
                                        st->out, cap, &st->count, lt, &ctl->fail, smem, &abytes, &items, &lbytes);
        if (a.stats) {                       // one add per CTA and step
            abytes = block_sum<NT, unsigned long long>(abytes, wt);
            items = block_sum<NT, unsigned long long>(items, wt);
            if (LW) lbytes = block_sum<NT, unsigned long long>(lbytes, wt);
            if (threadIdx.x == 0) {
                if (abytes) atomicAdd(a.stats, abytes);
                if (items) atomicAdd(a.stats + 1, items);
                if (lbytes) atomicAdd(a.stats + 2, lbytes);
            }
        }
        if (!grid_barrier(ctl, G)) return;
        if (__ldcg(&ctl->fail) & 1u) return;                  // long-row table full: a larger arena
        // ---- long rows through the candidate-slot tiles
        const uint64_t L = __ldcg(lt.count);
        if (L > 0 && !long_rows_join<NT, VT>(a, st, ctl, lt, L, st->S + ll.f_off,
                                             reinterpret_cast<int64_t *>(st->S + ll.part_off), ll.part_cap, cap,
                                             bsum, wt))
            return;
        if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) {      // survivors written (both models)
            const unsigned long long wbytes = 4ull * (uint64_t)(t + 1) * min((uint64_t)__ldcg(&st->count), cap);
            atomicAdd(a.stats, wbytes);
            if (LW) atomicAdd(a.stats + 2, wbytes);
        }
    }
}

__global__ void k_barrier_selftest(QueryCtl *ctl, unsigned expect) {
    // every CTA waits at a barrier that expects one CTA more than exist
    grid_barrier(ctl, expect);
}

std::once_flag g_join_attr_once[64];

StepDev step_dev(const gsi_graph *g, const JoinStep &s) {
    StepDev d;
    d.t = s.t;
    d.d = s.d;
    d.L = g->L;
    d.ulab = s.ulab;
    d.hom = s.hom;
    const uint32_t tmask = s.t >= 32 ? 0xffffffffu : ((1u << s.t) - 1u);
    d.inj = s.hom ? 0u : (s.inj & tmask);
    for (int i = 0; i < GSI_MAX_QUERY_VERTICES; ++i) {
        d.col[i] = i < s.d ? s.col[i] : 0;
        d.lab[i] = i < s.d ? s.lab[i] : 0;
    }
    return d;
}

}  // namespace

int64_t join_scan_scratch(uint64_t R) { return scan_blocks((int64_t)R) + 1 + ((int64_t)R + 1) / 2 + 1; }

gsi_status launch_join_scan(const gsi_graph *g, const int32_t *M, uint64_t R, const JoinStep &s, uint64_t *F,
                            uint64_t *scratch, cudaStream_t st) {
    // scratch: [scan block sums][per-row bounds as uint32]
    uint32_t *caps = reinterpret_cast<uint32_t *>(scratch + scan_blocks((int64_t)R) + 1);
    CapStoreProducer p1{M, g->off, g->cl, caps, (uint64_t)JOIN_ROW_WEIGHT, step_dev(g, s)};
    CapLoadProducer p2{caps, (uint64_t)JOIN_ROW_WEIGHT};
    GSI_CUDA_TRY(two_producer_scan(p1, p2, (int64_t)R, StoreWriter<uint64_t>{F}, scratch, st));
    return GSI_OK;
}

size_t join_smem(int rmax, int t, int d) {
    return (size_t)JOIN_NV * 8 + (size_t)(rmax + 1) * 8 + (size_t)rmax * 4 + (size_t)rmax * 2 * (d - 1) * 4 +
           (size_t)rmax * t * 4 + (size_t)JOIN_NV * 2;
}

gsi_status launch_partition(const uint64_t *F, uint64_t R, uint64_t total, int64_t *part, cudaStream_t st) {
    if (R == 0 || total == 0) return GSI_OK;
    const uint64_t ntiles = join_tiles(total);
    if (ntiles >= (1ull << 31)) {
        set_error("join: too many tiles in one launch");
        return GSI_EINVAL;
    }
    k_partition<<<(unsigned)((ntiles + 1 + 255) / 256), 256, 0, st>>>(F, (int64_t)R, total, (int64_t)ntiles, part);
    GSI_CUDA_TRY(cudaGetLastError());
    return GSI_OK;
}

gsi_status launch_join(const gsi_graph *g, const int32_t *M, uint64_t R, const JoinStep &s, const uint64_t *F,
                       uint64_t total, const int64_t *part, const uint32_t *cand, int32_t *out, uint64_t out_cap,
                       unsigned long long *out_count, int count_only, unsigned long long *stats, cudaStream_t st) {
    if (R == 0 || total == 0) return GSI_OK;
    const uint64_t ntiles = join_tiles(total);
    if (ntiles >= (1ull << 31)) {
        set_error("join: too many tiles in one launch");
        return GSI_EINVAL;
    }
    JoinArgs a;
    a.M = M; a.R = (int64_t)R; a.F = F; a.total = total; a.part = part;
    a.off = g->off; a.ci = g->ci; a.cl = g->cl; a.cand = cand;
    a.out = out; a.out_cap = out_cap; a.out_count = out_count; a.stats = stats;
    a.W = JOIN_ROW_WEIGHT;
    a.rmax = JOIN_NV / JOIN_ROW_WEIGHT + 2;
    a.count_only = count_only;
    a.s = step_dev(g, s);
    for (int i = 0; i <= GSI_MAX_QUERY_VERTICES; ++i) a.iperm[i] = i;
    for (int c = 0; c <= s.t; ++c) a.iperm[s.perm[c]] = c;
    size_t sm = join_smem(a.rmax, s.t, s.d);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {                 // once per device, safe across host threads
        cudaError_t e = cudaSuccess;
        std::call_once(g_join_attr_once[dev], [&e]() {
            e = cudaFuncSetAttribute(k_join<JOIN_NT, JOIN_VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024);
        });
        GSI_CUDA_TRY(e);
    }
    if (sm > 200 * 1024) {
        set_error("join: shared memory need exceeds 200 KB");
        return GSI_EINVAL;
    }
    k_join<JOIN_NT, JOIN_VT><<<(unsigned)ntiles, JOIN_NT, sm, st>>>(a);
    GSI_CUDA_TRY(cudaGetLastError());
    return GSI_OK;
}

JoinArgs make_join_args(const gsi_graph *g, const JoinStep &s, const uint32_t *cand, int count_only,
                        unsigned long long *stats) {
    JoinArgs a;
    std::memset(&a, 0, sizeof a);
    a.off = g->off; a.ci = g->ci; a.cl = g->cl; a.cand = cand;
    a.stats = stats;
    a.W = JOIN_ROW_WEIGHT;
    a.rmax = JOIN_NV / JOIN_ROW_WEIGHT + 2;
    a.count_only = count_only;
    a.s = step_dev(g, s);
    for (int i = 0; i <= GSI_MAX_QUERY_VERTICES; ++i) a.iperm[i] = i;
    for (int c = 0; c <= s.t; ++c) a.iperm[s.perm[c]] = c;
    return a;
}

size_t join_args_size() { return sizeof(JoinArgs); }

int query_memo_tables(const std::vector<JoinStep> &steps, int k) {
    int m = 0;
    for (int t = 1; t < k; ++t) m = std::max(m, std::min(steps[t].d, MEMO_EDGES));
    return m;
}

gsi_status query_coop_configs(const gsi_graph *g, const std::vector<JoinStep> &steps, int k, const uint32_t *bitmaps,
                              const int32_t *order, int count_only, unsigned long long *stats, uint64_t *memo, bool nodedup,
                              void *cfg_host, size_t *smem) {
    JoinArgs *cfg = static_cast<JoinArgs *>(cfg_host);
    std::memset(cfg, 0, sizeof(JoinArgs));
    size_t sm = 0;
    for (int t = 1; t < k; ++t) {
        const int co = (t == k - 1) && count_only;
        cfg[t] = make_join_args(g, steps[t], bitmaps + (uint64_t)order[t] * (uint64_t)g->nwords, co, stats);
        cfg[t].memo = nodedup ? nullptr : memo;
        cfg[t].memo_n = g->n;
        cfg[t].nodedup = nodedup ? 1 : 0;
        cfg[t].rmax = LONG_RMAX;             // the tiles of k_query see long rows only
        sm = std::max(sm, join_smem(cfg[t].rmax, steps[t].t, steps[t].d));
        sm = std::max(sm, rows_smem(JOIN_NT, steps[t].t));
    }
    if (sm > 200 * 1024) {
        set_error("join: shared memory need exceeds 200 KB");
        return GSI_EINVAL;
    }
    *smem = sm;
    return GSI_OK;
}

gsi_status launch_query_coop(const gsi_graph *g, int k, const uint32_t *seed_bitmap, size_t sm, void *cfg_dev,
                             DStep *dsteps, QueryCtl *ctl, unsigned long long *bsum, int *grid_out, bool listwise,
                             cudaStream_t st) {
    // the variant that also counts whole-list bytes costs registers: only on request
    const void *kern = listwise ? (const void *)k_query<JOIN_NT, JOIN_VT, true>
                                : (const void *)k_query<JOIN_NT, JOIN_VT, false>;
    int dev = 0;
    cudaGetDevice(&dev);
    // occupancy depends only on the dynamic shared memory: looked up once per
    // (device, size), as are the function attribute and the SM count
    static std::mutex mu;
    static std::map<std::tuple<int, size_t, bool>, int> occ;
    static int nsm[64];
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !nsm[dev]) {
            GSI_CUDA_TRY(cudaFuncSetAttribute(k_query<JOIN_NT, JOIN_VT, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            GSI_CUDA_TRY(cudaFuncSetAttribute(k_query<JOIN_NT, JOIN_VT, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            GSI_CUDA_TRY(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
        }
        auto it = occ.find({dev, sm, listwise});
        if (it != occ.end()) {
            per_sm = it->second;
        } else {
            GSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, JOIN_NT, sm));
            occ[{dev, sm, listwise}] = per_sm;
        }
    }
    if (per_sm < 1) {
        set_error("join: the query kernel does not fit on an SM");
        return GSI_EINVAL;
    }
    if (per_sm > 1024 / JOIN_NT) per_sm = 1024 / JOIN_NT;     // at most 32 warps per SM
    int grid = (dev >= 0 && dev < 64 ? nsm[dev] : 152) * per_sm;
    if (grid > QUERY_MAX_CTAS) grid = QUERY_MAX_CTAS;
    *grid_out = grid;
    const JoinArgs *cfgp = static_cast<const JoinArgs *>(cfg_dev);
    int64_t nwords = g->nwords;
    void *args[] = {(void *)&cfgp, (void *)&dsteps, (void *)&k, (void *)&ctl, (void *)&seed_bitmap, (void *)&nwords,
                    (void *)&bsum};
    GSI_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(JOIN_NT), args, sm, st));
    return GSI_OK;
}

gsi_status selftest_barrier_timeout(int dev, unsigned long long spin_limit, double *ms) {
    GSI_CUDA_TRY(cudaSetDevice(dev));
    QueryCtl *ctl = nullptr;
    GSI_CUDA_TRY(cudaMalloc(&ctl, sizeof(QueryCtl)));
    QueryCtl h;
    std::memset(&h, 0, sizeof h);
    h.spin_limit = spin_limit;
    gsi_status rc = GSI_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (cudaMemcpy(ctl, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) rc = GSI_ECUDA;
    const unsigned grid = 8;
    unsigned expect = grid + 1;
    void *args[] = {(void *)&ctl, (void *)&expect};
    if (rc == GSI_OK) {
        cudaEventRecord(e0, 0);
        if (cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(grid), dim3(JOIN_NT), args, 0, 0) !=
            cudaSuccess)
            rc = GSI_ECUDA;
        cudaEventRecord(e1, 0);
    }
    if (rc == GSI_OK && cudaMemcpy(&h, ctl, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) rc = GSI_ECUDA;
    float t = 0;
    if (rc == GSI_OK) cudaEventElapsedTime(&t, e0, e1);
    if (ms) *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ctl);
    if (rc != GSI_OK) {
        set_error("barrier self-test: launch or copy failed");
        return rc;
    }
    if (h.fail & 4u) {
        set_error("barrier self-test: the wait ran out as intended");
        return GSI_ETIMEOUT;
    }
    return GSI_OK;
}

}  // namespace gsi

// One join iteration (Sec. V, Algs. 3-4) as three launches:
//
//   1. scan   F[i] = sum_{r<i} (|N(m_r[u0'], l0)| + W): Alg. 4's exclusive
//             prefix sum of each row's output bound, plus W "row slots" per
//             row that pay for staging the row (load balancing, below).
//   2. part   for every tile of NV consecutive slots, its first row.
//   3. join   the fused kernel: one CTA per tile of NV slots.
//
// Work decomposition.  Instead of the paper's warp-per-row with a 4-layer
// balance scheme and dynamically launched child kernels (Sec. VI-A), every
// candidate w of N(m_i[u0'], l0) is one slot of a flat index space whose row
// offsets are F, and each CTA takes a fixed NV slots.  A hub row with 10^5
// candidates is spread over many CTAs; rows with one candidate are packed
// NV/W to a CTA.  The W per-row slots bound the rows one CTA stages, so its
// shared memory holds every row it touches.
//
// Per CTA (Sec. V "GPU-friendly set operation"):
//   * the partial matches m_i of its rows are staged in shared memory with
//     the located bounds of every neighbour list they need (small lists);
//   * slots read consecutive elements of N(v, l0) (coalesced medium list);
//   * C(u) is probed as a bitset, one 4-byte load per candidate (large list);
//   * set subtraction (w not in m_i) is checked against the staged row;
//   * the other linking edges test w in N(m_i[u_j'], l_j) by binary search
//     in the ascending list (the intersection), only for candidates that
//     survived the cheaper checks;
//   * survivors are compacted with one block-wide prefix sum and one global
//     atomic per CTA, then written once as rows of M' (Prealloc-Combine: the
//     join runs once; the output buffer is sized by F's total).
#include "internal.h"
#include "scan.cuh"

namespace gsi {
namespace {

struct CapProducer {
    const int32_t *M;
    int32_t t, c0, l0, L;
    const uint32_t *off;
    uint64_t W;
    __device__ uint64_t operator()(int64_t i) const {
        int32_t v = M[i * t + c0];
        uint64_t s = (uint64_t)(uint32_t)v * (uint64_t)L + (uint64_t)l0;
        return (uint64_t)(__ldg(off + s + 1) - __ldg(off + s)) + W;
    }
};

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

struct JoinArgs {
    const int32_t *M;
    int64_t R;
    const uint64_t *F;
    uint64_t total;
    const int64_t *part;
    const uint32_t *off;
    const int32_t *ci;
    const uint32_t *cand;
    int32_t *out;
    uint64_t out_cap;
    unsigned long long *out_count;
    unsigned long long *stats;
    int32_t t, d, L, W, rmax, count_only;
    int32_t col[GSI_MAX_QUERY_VERTICES];
    int32_t lab[GSI_MAX_QUERY_VERTICES];
    int32_t perm[GSI_MAX_QUERY_VERTICES + 1];
};

template <int NT, int VT>
__global__ void __launch_bounds__(NT) k_join(const __grid_constant__ JoinArgs a) {
    constexpr int NV = NT * VT;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long wt[NT / 32];
    __shared__ unsigned long long gbase_s;

    const int t = a.t, dm1 = a.d - 1;
    uint64_t *Fs = reinterpret_cast<uint64_t *>(smem);                 // rmax + 1
    uint32_t *base0 = reinterpret_cast<uint32_t *>(Fs + a.rmax + 1);    // rmax
    uint32_t *lst = base0 + a.rmax;                                     // rmax * 2 * dm1
    int32_t *rowv = reinterpret_cast<int32_t *>(lst + (size_t)a.rmax * 2 * dm1);   // rmax * t

    const uint64_t s0 = (uint64_t)blockIdx.x * NV;
    const uint64_t s1 = min(s0 + (uint64_t)NV, a.total);
    const int64_t r_lo = a.part[blockIdx.x];
    const int64_t r_hi = min(a.part[blockIdx.x + 1], a.R - 1);
    const int nr = (int)(r_hi - r_lo + 1);

    // ---- stage the tile's rows: values, first-edge list start, other lists
    unsigned long long bytes = 0;
    for (int lr = threadIdx.x; lr <= nr; lr += NT) Fs[lr] = a.F[r_lo + lr];
    for (int lr = threadIdx.x; lr < nr; lr += NT) {
        const int32_t *row = a.M + (r_lo + lr) * (int64_t)t;
        int32_t *rv = rowv + lr * t;
        for (int c = 0; c < t; ++c) rv[c] = row[c];
        uint64_t seg0 = (uint64_t)(uint32_t)rv[a.col[0]] * (uint64_t)a.L + (uint64_t)a.lab[0];
        base0[lr] = __ldg(a.off + seg0);
        uint64_t lsum = 0;
        for (int j = 1; j <= dm1; ++j) {
            uint64_t seg = (uint64_t)(uint32_t)rv[a.col[j]] * (uint64_t)a.L + (uint64_t)a.lab[j];
            uint32_t lo = __ldg(a.off + seg), hi = __ldg(a.off + seg + 1);
            lst[(lr * dm1 + (j - 1)) * 2] = lo;
            lst[(lr * dm1 + (j - 1)) * 2 + 1] = hi - lo;
            lsum += hi - lo;
        }
        if (a.stats && Fs[lr] >= s0) bytes += 4ull * t + 8ull * a.d + 4ull * lsum;   // row owned by this tile
    }
    __syncthreads();

    // ---- candidates: one slot per thread per round, consecutive slots per warp
    int32_t wv[VT];
    int32_t lrv[VT];
    unsigned okmask = 0;
    unsigned long long items = 0;
#pragma unroll
    for (int k = 0; k < VT; ++k) {
        const uint64_t s = s0 + (uint64_t)(k * NT + threadIdx.x);
        wv[k] = 0;
        lrv[k] = 0;
        if (s >= s1) continue;
        int lo = 0, hi = nr - 1;        // row of slot s: largest lr with Fs[lr] <= s
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (Fs[mid] <= s) lo = mid;
            else hi = mid - 1;
        }
        const int64_t p = (int64_t)(s - Fs[lo]) - a.W;
        if (p < 0) continue;            // a row-staging slot
        ++items;
        const int32_t w = __ldg(a.ci + (uint64_t)base0[lo] + (uint64_t)p);
        bool ok = (__ldg(a.cand + (w >> 5)) >> (w & 31)) & 1u;
        const int32_t *rv = rowv + lo * t;
        for (int c = 0; c < t && ok; ++c) ok = rv[c] != w;
        for (int j = 0; j < dm1 && ok; ++j) {
            const uint32_t *ls = lst + (lo * dm1 + j) * 2;
            ok = sorted_contains(a.ci + ls[0], ls[1], w);
        }
        wv[k] = w;
        lrv[k] = lo;
        if (ok) okmask |= 1u << k;
    }

    // ---- compaction: block prefix sum + one atomic per CTA, then write once
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan<NT, unsigned long long>(__popc(okmask), wt, &tot);
    if (threadIdx.x == 0) gbase_s = tot ? atomicAdd(a.out_count, tot) : 0ull;
    __syncthreads();
    if (!a.count_only) {
        uint64_t idx = gbase_s + ex;
#pragma unroll
        for (int k = 0; k < VT; ++k) {
            if (!((okmask >> k) & 1u)) continue;
            if (idx < a.out_cap) {
                int32_t *dst = a.out + idx * (uint64_t)(t + 1);
                const int32_t *rv = rowv + lrv[k] * t;
                for (int c = 0; c < t; ++c) dst[a.perm[c]] = rv[c];
                dst[a.perm[t]] = wv[k];
            }
            ++idx;
        }
    }
    if (a.stats) {
        bytes += 8ull * items;                                    // list element + bitmap probe
        if (!a.count_only) bytes += 4ull * (t + 1) * __popc(okmask);
        unsigned long long bsum = block_sum<NT, unsigned long long>(bytes, wt);
        unsigned long long isum = block_sum<NT, unsigned long long>(items, wt);
        if (threadIdx.x == 0) {
            atomicAdd(a.stats, bsum);
            atomicAdd(a.stats + 1, isum);
        }
    }
}

int g_smem_set[64];

}  // namespace

int64_t join_scan_scratch(uint64_t R) { return scan_blocks((int64_t)R) + 1; }

gsi_status launch_join_scan(const gsi_graph *g, const int32_t *M, uint64_t R, const JoinStep &s, uint64_t *F,
                            uint64_t *scratch, cudaStream_t st) {
    CapProducer p{M, s.t, s.col[0], s.lab[0], g->L, g->off, (uint64_t)JOIN_ROW_WEIGHT};
    GSI_CUDA_TRY(device_scan<uint64_t>(p, (int64_t)R, StoreWriter<uint64_t>{F}, scratch, st));
    return GSI_OK;
}

static size_t join_smem(int rmax, int t, int d) {
    return (size_t)(rmax + 1) * 8 + (size_t)rmax * 4 + (size_t)rmax * 2 * (d - 1) * 4 + (size_t)rmax * t * 4;
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
    a.off = g->off; a.ci = g->ci; a.cand = cand;
    a.out = out; a.out_cap = out_cap; a.out_count = out_count; a.stats = stats;
    a.t = s.t; a.d = s.d; a.L = g->L; a.W = JOIN_ROW_WEIGHT;
    a.rmax = JOIN_NV / JOIN_ROW_WEIGHT + 2;
    a.count_only = count_only;
    for (int i = 0; i < GSI_MAX_QUERY_VERTICES; ++i) {
        a.col[i] = i < s.d ? s.col[i] : 0;
        a.lab[i] = i < s.d ? s.lab[i] : 0;
    }
    for (int i = 0; i <= GSI_MAX_QUERY_VERTICES; ++i) a.perm[i] = i <= s.t ? s.perm[i] : i;
    size_t sm = join_smem(a.rmax, s.t, s.d);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !g_smem_set[dev]) {
        GSI_CUDA_TRY(cudaFuncSetAttribute(k_join<JOIN_NT, JOIN_VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        g_smem_set[dev] = 1;
    }
    if (sm > 200 * 1024) {
        set_error("join: shared memory need exceeds 200 KB");
        return GSI_EINVAL;
    }
    k_join<JOIN_NT, JOIN_VT><<<(unsigned)ntiles, JOIN_NT, sm, st>>>(a);
    GSI_CUDA_TRY(cudaGetLastError());
    return GSI_OK;
}

}  // namespace gsi

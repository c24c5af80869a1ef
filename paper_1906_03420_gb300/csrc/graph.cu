// Device graph build: label-partitioned CSR, label frequencies and the
// column-first signature table.
//
// Layout (Sec. IV, "basic representation" of the edge-label-partitioned
// graphs P(G,l)): every (vertex v, label l) pair owns one row-offset entry, so
// N(v,l) = ci[off[v*L+l] .. off[v*L+l+1]) is located with one 8-byte read.
// With the label counts of the target workloads (8-16 edge labels) this costs
// (L+1) * 4 bytes per vertex and replaces the paper's hashed PCSR groups,
// which exist to save that space when labels number in the tens of thousands.
// Each list N(v,l) is sorted by (label rank of the neighbour, neighbour id),
// with the label ranks kept in a parallel uint16 array cl: the neighbours of
// one vertex label form a contiguous, id-sorted sub-list, found by binary
// search on cl, and membership inside it is a binary search on ci.
//
// Signatures (Sec. III-A): N = 512 bits = 16 words per vertex, stored
// column-first (word w of vertex v at sig[w*n + v]) so a warp's 32 lanes read
// 32 consecutive words.  Word 0 is the vertex label itself (the K = 32 label
// bits).  Words 1..15 hold 240 two-bit groups: each (edge label, neighbour
// label) pair of v is hashed to a group whose state goes 00 -> 01 -> 11 as the
// first and second pair arrive.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "scan.cuh"

namespace gsi {
namespace {

constexpr int NT = 256;

enum : unsigned { BAD_ID = 1u, SELF_LOOP = 2u, NEG_LABEL = 4u, DUP_PAIR = 8u };

__global__ void k_validate(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                           const int32_t *__restrict__ elab, int64_t m, int32_t n, unsigned *flags, int *maxlab) {
    unsigned f = 0;
    int ml = -1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[e], b = dst[e], l = elab[e];
        if (a < 0 || a >= n || b < 0 || b >= n) f |= BAD_ID;
        if (a == b) f |= SELF_LOOP;
        if (l < 0) f |= NEG_LABEL;
        ml = max(ml, l);
    }
    f = __reduce_or_sync(FULL_MASK, f);
    ml = __reduce_max_sync(FULL_MASK, ml);
    if ((threadIdx.x & 31) == 0) {
        if (f) atomicOr(flags, f);
        atomicMax(maxlab, ml);
    }
}

__global__ void k_pair_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m, int nb,
                            uint64_t *__restrict__ keys) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = (uint32_t)src[e], b = (uint32_t)dst[e];
        keys[e] = a < b ? (a << nb) | b : (b << nb) | a;
    }
}

__global__ void k_adjacent_equal(const uint64_t *__restrict__ keys, int64_t n, unsigned *flags) {
    bool dup = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dup |= keys[i] == keys[i - 1];
    if (__any_sync(FULL_MASK, dup) && (threadIdx.x & 31) == 0) atomicOr(flags, (unsigned)DUP_PAIR);
}

// Dense rank of each vertex label (binary search in the sorted distinct labels).
__global__ void k_vertex_rank(const int32_t *__restrict__ vlab, int32_t n, const int32_t *__restrict__ uniq, int32_t LV,
                              uint16_t *__restrict__ rank) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = vlab[v], lo = 0, hi = LV - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi) >> 1;
            if (uniq[mid] < x) lo = mid + 1;
            else hi = mid;
        }
        rank[v] = (uint16_t)lo;
    }
}

// Directed entry keys: (((v*L + l) << lb | rank(neighbour)) << nb) | neighbour, two per edge.
__global__ void k_csr_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                           const int32_t *__restrict__ elab, const uint16_t *__restrict__ vrank, int64_t m, int32_t L,
                           int lb, int nb, uint64_t *__restrict__ keys) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = (uint32_t)src[e], b = (uint32_t)dst[e], l = (uint32_t)elab[e];
        keys[2 * e] = ((((a * (uint64_t)L + l) << lb) | vrank[b]) << nb) | b;
        keys[2 * e + 1] = ((((b * (uint64_t)L + l) << lb) | vrank[a]) << nb) | a;
    }
}

// From sorted keys: ci[p] = neighbour, cl[p] = its label rank, and off[s] =
// first position of segment s = v*L + l.
__global__ void k_csr_fill(const uint64_t *__restrict__ keys, int64_t n2, int lb, int nb, uint64_t nseg,
                           uint32_t *__restrict__ off, int32_t *__restrict__ ci, uint16_t *__restrict__ cl) {
    const uint64_t mask = (1ull << nb) - 1, lmask = (1ull << lb) - 1;
    const int sh = lb + nb;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n2; p += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[p];
        ci[p] = (int32_t)(k & mask);
        cl[p] = (uint16_t)((k >> nb) & lmask);
        uint64_t s = k >> sh;
        uint64_t prev = p == 0 ? 0 : (keys[p - 1] >> sh) + 1;
        for (uint64_t x = prev; x <= s; ++x) off[x] = (uint32_t)p;
        if (p == n2 - 1)
            for (uint64_t x = s + 1; x <= nseg; ++x) off[x] = (uint32_t)n2;
    }
}

__global__ void k_fill_u32(uint32_t *a, uint64_t n, uint32_t v) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_sig_labels(const int32_t *__restrict__ vlab, int32_t n, uint32_t *__restrict__ sig) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        sig[v] = (uint32_t)vlab[v];
}

// One (edge label, neighbour label) pair per directed entry.
__global__ void k_sig_pairs(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            const int32_t *__restrict__ elab, const int32_t *__restrict__ vlab, int64_t m, int32_t n,
                            uint32_t *__restrict__ sig) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i >> 1;
        int32_t v = (i & 1) ? dst[e] : src[e];
        int32_t w = (i & 1) ? src[e] : dst[e];
        uint32_t g = sig_group(elab[e], vlab[w]);
        uint32_t word = sig_word(g), bit = sig_bit(g);
        uint32_t *p = sig + (int64_t)word * n + v;
        uint32_t old = atomicOr(p, 1u << bit);
        if (old & (1u << bit)) atomicOr(p, 2u << bit);
    }
}

// Words 1..15 of every grouped position's vertex (zero for padding).
__global__ void k_group_sig(const uint32_t *__restrict__ sig, int32_t n, const int32_t *__restrict__ gperm,
                            int64_t np, uint32_t *__restrict__ gsig) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = gperm[p];
#pragma unroll
        for (int w = 1; w < GSI_SIG_WORDS; ++w) gsig[(int64_t)(w - 1) * np + p] = v >= 0 ? sig[(int64_t)w * n + v] : 0u;
    }
}

__global__ void k_label_hist(const int32_t *__restrict__ elab, int64_t m, int32_t L, unsigned long long *freq) {
    extern __shared__ unsigned long long h[];
    const bool local = L <= 4096;
    if (local)
        for (int i = threadIdx.x; i < L; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        if (local) atomicAdd(&h[elab[e]], 1ull);
        else atomicAdd(&freq[elab[e]], 1ull);
    }
    __syncthreads();
    if (local)
        for (int i = threadIdx.x; i < L; i += blockDim.x)
            if (h[i]) atomicAdd(&freq[i], h[i]);
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + NT - 1) / NT;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)b;
}

}  // namespace

gsi_status build_graph(gsi_graph *g, const int32_t *vlab, int32_t n, const int32_t *src, const int32_t *dst,
                       const int32_t *elab, int64_t m, cudaStream_t st) {
    if (n < 1 || m < 0) {
        set_error("gsi_graph_create: need n >= 1 and m >= 0");
        return GSI_EINVAL;
    }
    if (2 * m >= ((int64_t)1 << 32)) {
        set_error("gsi_graph_create: 2m must be below 2^32");
        return GSI_EINVAL;
    }
    if (m > 0 && (!src || !dst || !elab)) {
        set_error("gsi_graph_create: null edge arrays");
        return GSI_EINVAL;
    }
    if (!vlab) {
        set_error("gsi_graph_create: null vertex labels");
        return GSI_EINVAL;
    }
    cudaEvent_t e0, e1;
    GSI_CUDA_TRY(cudaEventCreate(&e0));
    GSI_CUDA_TRY(cudaEventCreate(&e1));
    GSI_CUDA_TRY(cudaEventRecord(e0, st));

    int32_t *d_vlab = nullptr, *d_src = nullptr, *d_dst = nullptr, *d_elab = nullptr;
    unsigned *d_flags = nullptr;
    int *d_maxlab = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync(&d_vlab, sizeof(int32_t) * (size_t)n, st));
    GSI_CUDA_TRY(cudaMallocAsync(&d_src, sizeof(int32_t) * (size_t)(m + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&d_dst, sizeof(int32_t) * (size_t)(m + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&d_elab, sizeof(int32_t) * (size_t)(m + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&d_flags, 16, st));
    d_maxlab = reinterpret_cast<int *>(d_flags + 1);
    GSI_CUDA_TRY(cudaMemcpyAsync(d_vlab, vlab, sizeof(int32_t) * (size_t)n, cudaMemcpyDefault, st));
    if (m > 0) {
        GSI_CUDA_TRY(cudaMemcpyAsync(d_src, src, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, st));
        GSI_CUDA_TRY(cudaMemcpyAsync(d_dst, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, st));
        GSI_CUDA_TRY(cudaMemcpyAsync(d_elab, elab, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, st));
    }
    GSI_CUDA_TRY(cudaMemsetAsync(d_flags, 0, 4, st));
    GSI_CUDA_TRY(cudaMemsetAsync(d_maxlab, 0xff, 4, st));   // -1
    auto cleanup_inputs = [&]() {
        cudaFreeAsync(d_vlab, st); cudaFreeAsync(d_src, st); cudaFreeAsync(d_dst, st);
        cudaFreeAsync(d_elab, st); cudaFreeAsync(d_flags, st);
    };
    if (m > 0) k_validate<<<grid_for(m), NT, 0, st>>>(d_src, d_dst, d_elab, m, n, d_flags, d_maxlab);
    unsigned h_flags[2] = {0, 0};
    GSI_CUDA_TRY(cudaMemcpyAsync(h_flags, d_flags, 8, cudaMemcpyDeviceToHost, st));
    GSI_CUDA_TRY(cudaStreamSynchronize(st));
    int maxlab = (int)h_flags[1];
    if (h_flags[0]) {
        cleanup_inputs();
        set_error(std::string("gsi_graph_create: ") + ((h_flags[0] & BAD_ID) ? "vertex id out of range " : "") +
                  ((h_flags[0] & SELF_LOOP) ? "self-loop " : "") + ((h_flags[0] & NEG_LABEL) ? "negative edge label" : ""));
        return GSI_EINVAL;
    }
    const int32_t L = maxlab < 0 ? 1 : maxlab + 1;
    // sorted distinct vertex labels (host): dense ranks for the sub-list order
    std::vector<int32_t> uniq;
    {
        int32_t mn = vlab[0], mx = vlab[0];
        for (int32_t v = 1; v < n; ++v) { mn = std::min(mn, vlab[v]); mx = std::max(mx, vlab[v]); }
        if ((int64_t)mx - (int64_t)mn < (1 << 24)) {
            std::vector<uint8_t> seen((size_t)((int64_t)mx - mn + 1), 0);
            for (int32_t v = 0; v < n; ++v) seen[(size_t)((int64_t)vlab[v] - mn)] = 1;
            for (size_t i = 0; i < seen.size(); ++i)
                if (seen[i]) uniq.push_back((int32_t)((int64_t)mn + (int64_t)i));
        } else {
            uniq.assign(vlab, vlab + n);
            std::sort(uniq.begin(), uniq.end());
            uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        }
    }
    if (uniq.size() > 65535) {
        cleanup_inputs();
        set_error("gsi_graph_create: more than 65535 distinct vertex labels");
        return GSI_EINVAL;
    }
    const int32_t LV = (int32_t)uniq.size();
    const int nb = ceil_log2_bits((uint64_t)(n > 1 ? n - 1 : 1));
    const int lb = ceil_log2_bits((uint64_t)(LV > 1 ? LV - 1 : 1));
    const uint64_t nseg = (uint64_t)n * (uint64_t)L;
    const int sb = ceil_log2_bits(nseg - 1);
    if (sb + lb + nb > 64 || nseg + 1 >= ((uint64_t)1 << 34)) {
        cleanup_inputs();
        set_error("gsi_graph_create: n * L * labels too large for the label-partitioned layout");
        return GSI_EINVAL;
    }

    // vertices grouped by label rank (host counting sort, ascending ids per
    // group, each group padded to a multiple of 32 positions)
    std::vector<int32_t> gperm;
    std::vector<int64_t> goff((size_t)LV + 1, 0);
    {
        std::vector<int32_t> rank((size_t)n);
        for (int32_t v = 0; v < n; ++v)
            rank[v] = (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), vlab[v]) - uniq.begin());
        std::vector<int64_t> cnt((size_t)LV, 0);
        for (int32_t v = 0; v < n; ++v) ++cnt[rank[v]];
        for (int32_t r = 0; r < LV; ++r) goff[r + 1] = goff[r] + (cnt[r] + 31) / 32 * 32;
        gperm.assign((size_t)goff[LV], -1);
        std::vector<int64_t> pos(goff.begin(), goff.end() - 1);
        for (int32_t v = 0; v < n; ++v) gperm[pos[rank[v]]++] = v;
    }

    // duplicate vertex pairs
    uint64_t *keys = nullptr, *tmp = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync(&keys, sizeof(uint64_t) * (size_t)(2 * m + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(uint64_t) * (size_t)(2 * m + 1), st));
    if (m > 1) {
        k_pair_keys<<<grid_for(m), NT, 0, st>>>(d_src, d_dst, m, nb, keys);
        GSI_TRY(radix_sort_u64(keys, tmp, m, 2 * nb, st));
        k_adjacent_equal<<<grid_for(m), NT, 0, st>>>(keys, m, d_flags);
        GSI_CUDA_TRY(cudaMemcpyAsync(h_flags, d_flags, 4, cudaMemcpyDeviceToHost, st));
        GSI_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_flags[0] & DUP_PAIR) {
            cudaFreeAsync(keys, st); cudaFreeAsync(tmp, st);
            cleanup_inputs();
            set_error("gsi_graph_create: a vertex pair appears more than once");
            return GSI_EINVAL;
        }
    }

    // CSR
    g->n = n; g->m = m; g->L = L; g->LV = LV; g->nwords = (n + 31) / 32;
    g->vlabels = uniq;
    GSI_CUDA_TRY(cudaMallocAsync(&g->off, sizeof(uint32_t) * (size_t)(nseg + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&g->ci, sizeof(int32_t) * (size_t)(2 * m + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&g->cl, sizeof(uint16_t) * (size_t)(2 * m + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&g->sig, sizeof(uint32_t) * (size_t)GSI_SIG_WORDS * (size_t)n, st));
    if (m > 0) {
        int32_t *d_uniq = nullptr;
        uint16_t *d_vrank = nullptr;
        GSI_CUDA_TRY(cudaMallocAsync(&d_uniq, sizeof(int32_t) * (size_t)LV, st));
        GSI_CUDA_TRY(cudaMallocAsync(&d_vrank, sizeof(uint16_t) * (size_t)n, st));
        GSI_CUDA_TRY(cudaMemcpyAsync(d_uniq, uniq.data(), sizeof(int32_t) * (size_t)LV, cudaMemcpyHostToDevice, st));
        k_vertex_rank<<<grid_for(n), NT, 0, st>>>(d_vlab, n, d_uniq, LV, d_vrank);
        k_csr_keys<<<grid_for(m), NT, 0, st>>>(d_src, d_dst, d_elab, d_vrank, m, L, lb, nb, keys);
        GSI_TRY(radix_sort_u64(keys, tmp, 2 * m, sb + lb + nb, st));
        k_csr_fill<<<grid_for(2 * m), NT, 0, st>>>(keys, 2 * m, lb, nb, nseg, g->off, g->ci, g->cl);
        cudaFreeAsync(d_uniq, st);
        cudaFreeAsync(d_vrank, st);
    } else {
        k_fill_u32<<<grid_for((int64_t)nseg + 1), NT, 0, st>>>(g->off, nseg + 1, 0u);
    }
    cudaFreeAsync(keys, st);
    cudaFreeAsync(tmp, st);

    // signatures
    GSI_CUDA_TRY(cudaMemsetAsync(g->sig, 0, sizeof(uint32_t) * (size_t)GSI_SIG_WORDS * (size_t)n, st));
    k_sig_labels<<<grid_for(n), NT, 0, st>>>(d_vlab, n, g->sig);
    if (m > 0) k_sig_pairs<<<grid_for(2 * m), NT, 0, st>>>(d_src, d_dst, d_elab, d_vlab, m, n, g->sig);

    // signatures grouped by label
    g->np = goff[LV];
    g->goff = goff;
    GSI_CUDA_TRY(cudaMallocAsync(&g->gperm, sizeof(int32_t) * (size_t)g->np, st));
    GSI_CUDA_TRY(cudaMallocAsync(&g->gsig, sizeof(uint32_t) * (size_t)(GSI_SIG_WORDS - 1) * (size_t)g->np, st));
    GSI_CUDA_TRY(cudaMemcpyAsync(g->gperm, gperm.data(), sizeof(int32_t) * (size_t)g->np, cudaMemcpyHostToDevice, st));
    k_group_sig<<<grid_for(g->np), NT, 0, st>>>(g->sig, n, g->gperm, g->np, g->gsig);

    // freq(l)
    unsigned long long *d_freq = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync(&d_freq, sizeof(unsigned long long) * (size_t)L, st));
    GSI_CUDA_TRY(cudaMemsetAsync(d_freq, 0, sizeof(unsigned long long) * (size_t)L, st));
    if (m > 0) {
        size_t sm = L <= 4096 ? sizeof(unsigned long long) * (size_t)L : 0;
        k_label_hist<<<grid_for(m), NT, sm, st>>>(d_elab, m, L, d_freq);
    }
    g->freq.assign((size_t)L, 0);
    GSI_CUDA_TRY(cudaMemcpyAsync(g->freq.data(), d_freq, sizeof(uint64_t) * (size_t)L, cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(d_freq, st);
    cleanup_inputs();
    GSI_CUDA_TRY(cudaGetLastError());
    GSI_CUDA_TRY(cudaEventRecord(e1, st));
    GSI_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->build_ms = ms;
    g->device_bytes = sizeof(uint32_t) * (nseg + 1) + sizeof(int32_t) * (uint64_t)(2 * m + 1) +
                      sizeof(uint16_t) * (uint64_t)(2 * m + 1) + sizeof(uint32_t) * GSI_SIG_WORDS * (uint64_t)n +
                      sizeof(uint32_t) * GSI_SIG_WORDS * (uint64_t)g->np;
    return GSI_OK;
}

}  // namespace gsi

// Filtering phase (Sec. III-A) and the seed of the intermediate table.
//
// One pass over the column-first signature table tests every query vertex at
// once: a warp takes 32 consecutive data vertices, reads word 0 (the label) of
// each, and only lanes whose label equals some query vertex's label read words
// 1..15.  For each query vertex u the warp's 32 verdicts become one bitmap
// word of C(u) through __ballot_sync, so C(u) is written directly in the
// bitset form the join probes (Sec. V, "GPU-friendly set operation").
#include <vector>

#include "internal.h"
#include "scan.cuh"

namespace gsi {
namespace {

constexpr int FNT = 256;

struct FilterArgs {
    const uint32_t *sig;
    int32_t n;
    int32_t k;
    int32_t nwords;
    uint32_t *bitmaps;
    unsigned long long *counts;
    uint32_t q[GSI_MAX_QUERY_VERTICES][GSI_SIG_WORDS];
};

__global__ void __launch_bounds__(FNT) k_filter(const __grid_constant__ FilterArgs a) {
    __shared__ uint32_t qs[GSI_MAX_QUERY_VERTICES][GSI_SIG_WORDS];
    __shared__ unsigned long long cnt[GSI_MAX_QUERY_VERTICES];
    for (int i = threadIdx.x; i < a.k * GSI_SIG_WORDS; i += FNT) qs[i / GSI_SIG_WORDS][i % GSI_SIG_WORDS] =
        a.q[i / GSI_SIG_WORDS][i % GSI_SIG_WORDS];
    if (threadIdx.x < GSI_MAX_QUERY_VERTICES) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (FNT / 32);
    unsigned long long mycnt = 0;     // lane u < k accumulates C(u)'s count
    for (int64_t grp = (int64_t)blockIdx.x * (FNT / 32) + (threadIdx.x >> 5); grp < a.nwords; grp += warps) {
        const int64_t v = grp * 32 + lane;
        const bool valid = v < a.n;
        const uint32_t lab = valid ? __ldg(a.sig + v) : 0u;
        uint32_t match = 0;
        for (int u = 0; u < a.k; ++u) match |= (valid && lab == qs[u][0]) ? (1u << u) : 0u;
        uint32_t w[GSI_SIG_WORDS];
#pragma unroll
        for (int j = 1; j < GSI_SIG_WORDS; ++j) w[j] = match ? __ldg(a.sig + (int64_t)j * a.n + v) : 0u;
        for (int u = 0; u < a.k; ++u) {
            bool pass = (match >> u) & 1u;
#pragma unroll
            for (int j = 1; j < GSI_SIG_WORDS; ++j) pass = pass && ((w[j] & qs[u][j]) == qs[u][j]);
            unsigned b = __ballot_sync(FULL_MASK, pass);
            if (lane == 0) a.bitmaps[(int64_t)u * a.nwords + grp] = b;
            if (lane == u) mycnt += __popc(b);
        }
    }
    if (lane < a.k && mycnt) atomicAdd(&cnt[lane], mycnt);
    __syncthreads();
    if (threadIdx.x < a.k && cnt[threadIdx.x]) atomicAdd(&a.counts[threadIdx.x], cnt[threadIdx.x]);
}

// All query vertices of a batch in one pass over the signature table: each
// warp reads the 16 words of its 32 data vertices once and tests every query
// vertex against them.  Bitmaps must be zeroed; only non-empty words are
// written.
__global__ void __launch_bounds__(FNT) k_filter_batch(const uint32_t *__restrict__ sig, int32_t n, int32_t nwords,
                                                      const uint32_t *__restrict__ qsig, int32_t nqv,
                                                      uint32_t *__restrict__ bitmaps,
                                                      unsigned long long *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (FNT / 32);
    for (int64_t grp = (int64_t)blockIdx.x * (FNT / 32) + (threadIdx.x >> 5); grp < nwords; grp += warps) {
        const int64_t v = grp * 32 + lane;
        const bool valid = v < n;
        const uint32_t lab = valid ? __ldg(sig + v) : 0xffffffffu;
        uint32_t w[GSI_SIG_WORDS];
#pragma unroll
        for (int j = 1; j < GSI_SIG_WORDS; ++j) w[j] = valid ? __ldg(sig + (int64_t)j * n + v) : 0u;
        for (int32_t u = 0; u < nqv; ++u) {
            const uint32_t *q = qsig + (int64_t)u * GSI_SIG_WORDS;
            const uint32_t ql = __ldg(q);
            bool pass = valid && lab == ql;
            if (!__any_sync(FULL_MASK, pass)) continue;
#pragma unroll
            for (int j = 1; j < GSI_SIG_WORDS; ++j) {
                const uint32_t qw = __ldg(q + j);
                pass = pass && ((w[j] & qw) == qw);
            }
            const unsigned b = __ballot_sync(FULL_MASK, pass);
            if (b && lane == 0) {
                bitmaps[(int64_t)u * nwords + grp] = b;
                atomicAdd(&counts[u], (unsigned long long)__popc(b));
            }
        }
    }
}

struct PopcProducer {
    const uint32_t *bm;
    __device__ uint32_t operator()(int64_t i) const { return __popc(bm[i]); }
};
struct SeedWriter {
    const uint32_t *bm;
    int64_t nwords;
    int32_t *out;
    __device__ void operator()(int64_t i, uint32_t pos) const {
        if (i >= nwords) return;
        uint32_t b = bm[i];
        while (b) {
            int bit = __ffs(b) - 1;
            out[pos++] = (int32_t)(i * 32 + bit);
            b &= b - 1;
        }
    }
};

}  // namespace

void query_signatures(const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                      const int32_t *qelab, int32_t qm, QuerySig *out) {
    out->k = k;
    uint32_t counts[GSI_MAX_QUERY_VERTICES][GSI_SIG_GROUPS];
    for (int u = 0; u < k; ++u)
        for (int gidx = 0; gidx < GSI_SIG_GROUPS; ++gidx) counts[u][gidx] = 0;
    for (int e = 0; e < qm; ++e) {
        int a = qsrc[e], b = qdst[e];
        counts[a][sig_group(qelab[e], qvlab[b])]++;
        counts[b][sig_group(qelab[e], qvlab[a])]++;
    }
    for (int u = 0; u < k; ++u) {
        for (int w = 0; w < GSI_SIG_WORDS; ++w) out->sig[u][w] = 0;
        out->sig[u][0] = (uint32_t)qvlab[u];
        for (uint32_t gidx = 0; gidx < GSI_SIG_GROUPS; ++gidx) {
            if (counts[u][gidx] >= 1) out->sig[u][sig_word(gidx)] |= 1u << sig_bit(gidx);
            if (counts[u][gidx] >= 2) out->sig[u][sig_word(gidx)] |= 2u << sig_bit(gidx);
        }
    }
}

gsi_status launch_filter(const gsi_graph *g, const QuerySig &q, uint32_t *bitmaps, unsigned long long *counts,
                         cudaStream_t st) {
    FilterArgs a;
    a.sig = g->sig;
    a.n = g->n;
    a.k = q.k;
    a.nwords = g->nwords;
    a.bitmaps = bitmaps;
    a.counts = counts;
    for (int u = 0; u < GSI_MAX_QUERY_VERTICES; ++u)
        for (int w = 0; w < GSI_SIG_WORDS; ++w) a.q[u][w] = u < q.k ? q.sig[u][w] : 0u;
    GSI_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)q.k, st));
    int64_t blocks = ((int64_t)g->nwords + (FNT / 32) - 1) / (FNT / 32);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_filter<<<(unsigned)blocks, FNT, 0, st>>>(a);
    GSI_CUDA_TRY(cudaGetLastError());
    return GSI_OK;
}

gsi_status launch_filter_batch(const gsi_graph *g, const std::vector<QuerySig> &qs, uint32_t *bitmaps,
                               unsigned long long *counts, cudaStream_t st) {
    std::vector<uint32_t> flat;
    for (const QuerySig &q : qs)
        for (int u = 0; u < q.k; ++u) flat.insert(flat.end(), q.sig[u], q.sig[u] + GSI_SIG_WORDS);
    const int32_t nqv = (int32_t)(flat.size() / GSI_SIG_WORDS);
    if (nqv == 0) return GSI_OK;
    uint32_t *d_q = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync(&d_q, flat.size() * 4, st));
    GSI_CUDA_TRY(cudaMemcpyAsync(d_q, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice, st));
    GSI_CUDA_TRY(cudaMemsetAsync(bitmaps, 0, (size_t)nqv * (size_t)g->nwords * 4, st));
    GSI_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)nqv * 8, st));
    int64_t blocks = ((int64_t)g->nwords + (FNT / 32) - 1) / (FNT / 32);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_filter_batch<<<(unsigned)blocks, FNT, 0, st>>>(g->sig, g->n, g->nwords, d_q, nqv, bitmaps, counts);
    GSI_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(d_q, st);
    return GSI_OK;
}

int64_t seed_scratch_words(const gsi_graph *g) { return scan_blocks(g->nwords) + 1; }

gsi_status launch_seed(const gsi_graph *g, const uint32_t *bitmap, int32_t *out, uint32_t *scratch,
                       cudaStream_t st) {
    GSI_CUDA_TRY(device_scan<uint32_t>(PopcProducer{bitmap}, g->nwords, SeedWriter{bitmap, g->nwords, out}, scratch,
                                       st));
    return GSI_OK;
}

}  // namespace gsi

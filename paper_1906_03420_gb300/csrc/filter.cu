// Filtering phase (Sec. III-A) and the seed of the intermediate table.
//
// The filter reads the signature table in its label-grouped copy (vertex ids
// of each label in ascending order, groups padded to whole warps), so a warp
// holds 32 vertices of one label and is only visited when some query vertex
// of the call carries that label: the label test of Sec. III-A becomes the
// choice of warps, and the remaining 15 words decide S(v) & S(u) == S(u) for
// the query vertices of that label only.  One call serves every query vertex
// of a query or of a whole batch.  Each verdict becomes a bit of the bitmap
// C(u) (the set form the join probes, Sec. V): lanes whose vertices share a
// bitmap word (consecutive, as ids ascend) OR their bits together and the
// last of them sets them with one atomicOr.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"
#include "scan.cuh"

namespace gsi {
namespace {

constexpr int FNT = 256;

// meta: qid[nqv] (bitmap / counter index of sorted query vertex s),
// gstart[ngroups + 1] (query vertices of group g), wbeg[ngroups] (first warp
// of the group's label), wcum[ngroups + 1] (prefix of the groups' warps).
__global__ void __launch_bounds__(FNT) k_filter_groups(const int32_t *__restrict__ gperm,
                                                       const uint32_t *__restrict__ gsig, int64_t np,
                                                       const uint32_t *__restrict__ qsig,
                                                       const int32_t *__restrict__ meta, int32_t ngroups,
                                                       int32_t nqv, int32_t shared_counts, int32_t nwords,
                                                       uint32_t *__restrict__ bitmaps,
                                                       unsigned long long *__restrict__ counts) {
    extern __shared__ uint32_t scnt[];
    const int32_t *qid = meta;
    const int32_t *gstart = qid + nqv;
    const int32_t *wbeg = gstart + ngroups + 1;
    const int32_t *wcum = wbeg + ngroups;
    if (shared_counts)
        for (int32_t s = threadIdx.x; s < nqv; s += FNT) scnt[s] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t total = __ldg(wcum + ngroups);
    const int64_t stride = (int64_t)gridDim.x * (FNT / 32);
    for (int64_t aw = (int64_t)blockIdx.x * (FNT / 32) + (threadIdx.x >> 5); aw < total; aw += stride) {
        int lo = 0, hi = ngroups - 1;                  // the group whose warps hold aw
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(wcum + mid) <= aw) lo = mid;
            else hi = mid - 1;
        }
        const int g = lo;
        const int64_t p = ((int64_t)__ldg(wbeg + g) + (aw - __ldg(wcum + g))) * 32 + lane;
        const int32_t v = __ldg(gperm + p);
        uint32_t x[GSI_SIG_WORDS - 1];
#pragma unroll
        for (int j = 0; j < GSI_SIG_WORDS - 1; ++j) x[j] = __ldg(gsig + (int64_t)j * np + p);
        const int32_t word = v >= 0 ? (v >> 5) : -1;
        const unsigned run = __match_any_sync(FULL_MASK, word);   // lanes sharing my bitmap word
        const int first = __ffs(run) - 1;
        const bool last = 31 - __clz(run) == lane;
        const int32_t s1 = __ldg(gstart + g + 1);
        for (int32_t s = __ldg(gstart + g); s < s1; ++s) {
            const uint32_t *q = qsig + (int64_t)s * GSI_SIG_WORDS;
            bool pass = v >= 0;
#pragma unroll
            for (int j = 1; j < GSI_SIG_WORDS; ++j) {
                const uint32_t qw = __ldg(q + j);
                pass = pass && ((x[j - 1] & qw) == qw);
            }
            uint32_t bit = pass ? 1u << (v & 31) : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, bit, o);
                if (lane - o >= first) bit |= y;
            }
            if (last && bit) atomicOr(&bitmaps[(int64_t)__ldg(qid + s) * nwords + word], bit);
            const unsigned b = __ballot_sync(FULL_MASK, pass);
            if (b && lane == 0) {
                if (shared_counts) atomicAdd(&scnt[s], (uint32_t)__popc(b));
                else atomicAdd(&counts[__ldg(qid + s)], (unsigned long long)__popc(b));
            }
        }
    }
    if (shared_counts) {
        __syncthreads();
        for (int32_t s = threadIdx.x; s < nqv; s += FNT)
            if (scnt[s]) atomicAdd(&counts[__ldg(qid + s)], (unsigned long long)scnt[s]);
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
                      const int32_t *qelab, int32_t qm, QuerySig *out, bool hom) {
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
            if (counts[u][gidx] >= 2 && !hom) out->sig[u][sig_word(gidx)] |= 2u << sig_bit(gidx);
        }
    }
}

// Groups the query vertices in sigs (bitmap / counter index = position in
// sigs) by label and uploads their signatures with the group table; a group
// whose label no data vertex carries is dropped (its C(u) stays empty).
gsi_status filter_plan(const gsi_graph *g, const std::vector<const uint32_t *> &sigs, FilterPlan *fp,
                       cudaStream_t st) {
    *fp = FilterPlan();
    const int32_t nqv = (int32_t)sigs.size();
    fp->nqv = nqv;
    if (nqv == 0) return GSI_OK;
    std::vector<int32_t> perm((size_t)nqv);
    for (int32_t i = 0; i < nqv; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return sigs[a][0] < sigs[b][0]; });
    std::vector<uint32_t> flat;
    std::vector<int32_t> qid, gstart, wbeg, wcum;
    flat.reserve((size_t)nqv * GSI_SIG_WORDS);
    int64_t warps = 0;
    for (int32_t i = 0; i < nqv;) {
        int32_t j = i;
        while (j < nqv && sigs[perm[j]][0] == sigs[perm[i]][0]) ++j;
        const int32_t r = g->label_rank((int32_t)sigs[perm[i]][0]);
        if (r >= 0 && g->goff[r + 1] > g->goff[r]) {
            gstart.push_back((int32_t)qid.size());
            wbeg.push_back((int32_t)(g->goff[r] / 32));
            wcum.push_back((int32_t)warps);
            warps += (g->goff[r + 1] - g->goff[r]) / 32;
            for (int32_t t = i; t < j; ++t) {
                qid.push_back(perm[t]);
                flat.insert(flat.end(), sigs[perm[t]], sigs[perm[t]] + GSI_SIG_WORDS);
            }
        }
        i = j;
    }
    // up to 96 KB of per-CTA counters (set once per device, outside any
    // stream capture)
    {
        static std::once_flag once[64];
        int dev = 0;
        cudaGetDevice(&dev);
        cudaError_t e = cudaSuccess;
        if (dev >= 0 && dev < 64)
            std::call_once(once[dev], [&e]() {
                e = cudaFuncSetAttribute(k_filter_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            });
        GSI_CUDA_TRY(e);
    }
    fp->ngroups = (int32_t)wbeg.size();
    fp->nq = (int32_t)qid.size();
    fp->warps = warps;
    if (fp->ngroups == 0) return GSI_OK;
    gstart.push_back(fp->nq);
    wcum.push_back((int32_t)warps);
    std::vector<int32_t> meta;
    meta.reserve(qid.size() + gstart.size() + wbeg.size() + wcum.size());
    meta.insert(meta.end(), qid.begin(), qid.end());
    meta.insert(meta.end(), gstart.begin(), gstart.end());
    meta.insert(meta.end(), wbeg.begin(), wbeg.end());
    meta.insert(meta.end(), wcum.begin(), wcum.end());
    const size_t qbytes = flat.size() * 4;
    GSI_CUDA_TRY(cudaMallocAsync(&fp->d_q, qbytes + meta.size() * 4, st));
    fp->d_meta = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(fp->d_q) + qbytes);
    GSI_CUDA_TRY(cudaMemcpyAsync(fp->d_q, flat.data(), qbytes, cudaMemcpyHostToDevice, st));
    GSI_CUDA_TRY(cudaMemcpyAsync(fp->d_meta, meta.data(), meta.size() * 4, cudaMemcpyHostToDevice, st));
    return GSI_OK;
}

// Zeroes the bitmaps and counters, then runs the filter kernel: stream work
// only (no host synchronisation, no allocation), so it can be captured.
gsi_status filter_enqueue(const gsi_graph *g, const FilterPlan &fp, uint32_t *bitmaps, unsigned long long *counts,
                          cudaStream_t st) {
    if (fp.nqv == 0) return GSI_OK;
    GSI_CUDA_TRY(cudaMemsetAsync(bitmaps, 0, (size_t)fp.nqv * (size_t)g->nwords * 4, st));
    GSI_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)fp.nqv * 8, st));
    if (fp.ngroups == 0) return GSI_OK;
    int64_t blocks = (fp.warps + (FNT / 32) - 1) / (FNT / 32);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    // per-CTA counters in shared memory when they fit (else global atomics)
    const size_t smem = (size_t)fp.nq * 4;
    const int shared_counts = smem <= 96 * 1024 ? 1 : 0;
    k_filter_groups<<<(unsigned)blocks, FNT, shared_counts ? smem : 0, st>>>(
        g->gperm, g->gsig, g->np, fp.d_q, fp.d_meta, fp.ngroups, fp.nq, shared_counts, g->nwords, bitmaps, counts);
    GSI_CUDA_TRY(cudaGetLastError());
    return GSI_OK;
}

void filter_plan_free(FilterPlan &fp, cudaStream_t st) {
    if (fp.d_q) cudaFreeAsync(fp.d_q, st);
    fp = FilterPlan();
}

static gsi_status launch_filter_groups(const gsi_graph *g, const std::vector<const uint32_t *> &sigs,
                                       uint32_t *bitmaps, unsigned long long *counts, cudaStream_t st) {
    FilterPlan fp;
    gsi_status rc = filter_plan(g, sigs, &fp, st);
    if (rc == GSI_OK) rc = filter_enqueue(g, fp, bitmaps, counts, st);
    filter_plan_free(fp, st);
    return rc;
}

gsi_status launch_filter(const gsi_graph *g, const QuerySig &q, uint32_t *bitmaps, unsigned long long *counts,
                         cudaStream_t st) {
    std::vector<const uint32_t *> sigs;
    for (int u = 0; u < q.k; ++u) sigs.push_back(q.sig[u]);
    return launch_filter_groups(g, sigs, bitmaps, counts, st);
}

gsi_status launch_filter_batch(const gsi_graph *g, const std::vector<QuerySig> &qs, uint32_t *bitmaps,
                               unsigned long long *counts, cudaStream_t st) {
    std::vector<const uint32_t *> sigs;
    for (const QuerySig &q : qs)
        for (int u = 0; u < q.k; ++u) sigs.push_back(q.sig[u]);
    return launch_filter_groups(g, sigs, bitmaps, counts, st);
}

// Bytes the filter must move for these query vertices: the grouped words of
// every label they carry (ids and 15 signature words) and their bitmaps.
uint64_t filter_alg_bytes(const gsi_graph *g, const std::vector<int32_t> &labels) {
    std::vector<int32_t> l(labels);
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
    uint64_t b = 0;
    for (int32_t x : l) {
        const int32_t r = g->label_rank(x);
        if (r >= 0) b += (uint64_t)(g->goff[r + 1] - g->goff[r]) * 4ull * GSI_SIG_WORDS;
    }
    return b + (uint64_t)labels.size() * (uint64_t)g->nwords * 4ull;
}

int64_t seed_scratch_words(const gsi_graph *g) { return scan_blocks(g->nwords) + 1; }

gsi_status launch_seed(const gsi_graph *g, const uint32_t *bitmap, int32_t *out, uint32_t *scratch,
                       cudaStream_t st) {
    GSI_CUDA_TRY(device_scan<uint32_t>(PopcProducer{bitmap}, g->nwords, SeedWriter{bitmap, g->nwords, out}, scratch,
                                       st));
    return GSI_OK;
}

}  // namespace gsi

// Declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gsi.h"

struct gsi_graph {
    int device = 0;
    int32_t n = 0;
    int64_t m = 0;
    int32_t L = 1;              // edge labels 0..L-1
    int32_t LV = 1;             // distinct vertex labels
    int32_t nwords = 0;         // ceil(n / 32): words of one candidate bitmap
    uint32_t *off = nullptr;    // [n*L + 1]
    int32_t *ci = nullptr;      // [2m], each N(v,l) sorted by (label rank of neighbour, id)
    uint16_t *cl = nullptr;     // [2m], label rank of ci[p]
    uint32_t *sig = nullptr;    // [16 * n], column-first
    // the same signatures grouped by vertex label: gperm holds the vertex ids
    // of each label rank in ascending order, every group padded with -1 to a
    // multiple of 32 positions (goff: first position of each group); gsig holds
    // words 1..15 of gperm[p] at gsig[(w - 1) * np + p] (0 for padding)
    int32_t *gperm = nullptr;   // [np]
    uint32_t *gsig = nullptr;   // [15 * np]
    int64_t np = 0;
    std::vector<int64_t> goff;  // [LV + 1]
    std::vector<uint64_t> freq; // [L]
    std::vector<int32_t> vlabels;   // sorted distinct vertex labels; rank = index
    int32_t label_rank(int32_t label) const;   // -1 if no vertex carries it
    uint64_t device_bytes = 0;
    double build_ms = 0;
};

namespace gsi {

// ------------------------------------------------------------------ sort
// Ascending LSD radix sort of n keys over their low `bits` bits.  keys and
// tmp hold n keys each; the result ends in keys.  Scratch is allocated
// stream-ordered.
gsi_status radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, cudaStream_t st);

// ----------------------------------------------------------------- graph
gsi_status build_graph(gsi_graph *g, const int32_t *vlab, int32_t n, const int32_t *src, const int32_t *dst,
                       const int32_t *elab, int64_t m, cudaStream_t st);

// ---------------------------------------------------------------- filter
struct QuerySig {
    int32_t k = 0;
    uint32_t sig[GSI_MAX_QUERY_VERTICES][GSI_SIG_WORDS];
};
// hom: homomorphism semantics keeps only the "at least one" group states.
void query_signatures(const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                      const int32_t *qelab, int32_t qm, QuerySig *out, bool hom = false);
// bitmaps: device uint32[k][nwords]; counts: device unsigned long long[k] (both zeroed here).
gsi_status launch_filter(const gsi_graph *g, const QuerySig &q, uint32_t *bitmaps, unsigned long long *counts,
                         cudaStream_t st);
// Every query vertex of a batch in one pass: bitmaps [sum k][nwords] and
// counts [sum k] in query order (zeroed here).
gsi_status launch_filter_batch(const gsi_graph *g, const std::vector<QuerySig> &qs, uint32_t *bitmaps,
                               unsigned long long *counts, cudaStream_t st);
// A filter call split in two: filter_plan groups the query vertices by label
// and uploads their signatures (host work, stream-ordered allocation);
// filter_enqueue zeroes bitmaps [nqv][nwords] and counters [nqv] and runs the
// kernel (stream work only: capturable into a CUDA graph).
struct FilterPlan {
    uint32_t *d_q = nullptr;    // grouped signatures, then the group table
    int32_t *d_meta = nullptr;
    int32_t nqv = 0, nq = 0, ngroups = 0;
    int64_t warps = 0;
};
gsi_status filter_plan(const gsi_graph *g, const std::vector<const uint32_t *> &sigs, FilterPlan *fp,
                       cudaStream_t st);
gsi_status filter_enqueue(const gsi_graph *g, const FilterPlan &fp, uint32_t *bitmaps, unsigned long long *counts,
                          cudaStream_t st);
void filter_plan_free(FilterPlan &fp, cudaStream_t st);
// Algorithmic bytes of one filter call over query vertices with these labels.
uint64_t filter_alg_bytes(const gsi_graph *g, const std::vector<int32_t> &labels);
// Compact the bitmap of C(u) into the int32 list out (ascending); scratch: uint32[scan_blocks+1].
gsi_status launch_seed(const gsi_graph *g, const uint32_t *bitmap, int32_t *out, uint32_t *scratch,
                       cudaStream_t st);
int64_t seed_scratch_words(const gsi_graph *g);

// ------------------------------------------------------------------ join
struct JoinStep {
    int32_t t = 0;                       // columns of M
    int32_t ulab = 0;                    // label rank of the new query vertex
    int32_t d = 0;                       // linking edges; [0] is e0 (Alg. 4)
    int32_t col[GSI_MAX_QUERY_VERTICES];
    int32_t lab[GSI_MAX_QUERY_VERTICES];
    int32_t perm[GSI_MAX_QUERY_VERTICES + 1];   // output position of each column
    int32_t hom = 0;                     // 1: homomorphism (no set subtraction, Sec. VII-A)
    uint32_t inj = 0xffffffffu;          // columns whose query vertex has u's label (set subtraction)
};

constexpr int JOIN_NT = 256;
constexpr int JOIN_VT = 4;
constexpr int JOIN_NV = JOIN_NT * JOIN_VT;
constexpr int JOIN_ROW_WEIGHT = 2;      // slots charged per row (row staging work)

// Exclusive scan over rows of (cap_i + W): F[0..R], F[R] = total slots, where
// cap_i is the shortest label sub-list of row i's linking lists.
gsi_status launch_join_scan(const gsi_graph *g, const int32_t *M, uint64_t R, const JoinStep &s, uint64_t *F,
                            uint64_t *scratch, cudaStream_t st);
int64_t join_scan_scratch(uint64_t R);
// part[b] = first row of slot tile b, for b in [0, join_tiles(total)]; total = F[R].
gsi_status launch_partition(const uint64_t *F, uint64_t R, uint64_t total, int64_t *part, cudaStream_t st);
// The fused join kernel.  out_count (device) is incremented by the number of
// survivors; stats (device, nullable): [0] algorithmic bytes, [1] candidates.
gsi_status launch_join(const gsi_graph *g, const int32_t *M, uint64_t R, const JoinStep &s, const uint64_t *F,
                       uint64_t total, const int64_t *part, const uint32_t *cand, int32_t *out, uint64_t out_cap,
                       unsigned long long *out_count, int count_only, unsigned long long *stats, cudaStream_t st);
inline uint64_t join_tiles(uint64_t total) { return (total + JOIN_NV - 1) / JOIN_NV; }

// One join step of a cooperative query launch (see join.cu): the host sets
// the regions, the device the sizes.
struct DStep {
    // set by the host
    const int32_t *M;                  // input table (t columns)
    int32_t *out;                      // output table region
    uint64_t out_bytes;                // bytes of the output region
    uint64_t row_cap;                  // output rows allowed (0 = no limit)
    uint64_t *S;                       // scratch region: the long-row table (rows, bound
                                       // records), its slot offsets F and tile partition
    uint64_t S_words;
    int32_t t, count_only;
    // set on the device
    unsigned long long count;          // survivors (exact even past out_cap); [0]: seed size
    unsigned long long next_tile;
    unsigned long long nlong;          // rows set aside for the slot tiles (bound above SHORT_MAX)
    uint64_t R, total, ntiles, out_cap;
};

// Grid-barrier and status words of one cooperative query launch.
struct QueryCtl {
    unsigned bar_count, bar_gen;
    unsigned fail;        // 1 scratch too small (or a sub-list too long for a bound record),
                          // 2 table overflow, 4 barrier wait gave up
    unsigned pad;
    unsigned long long spin_limit;   // sleeps before a barrier wait gives up (0 = default)
};
constexpr int QUERY_MAX_CTAS = 2048;
size_t join_args_size();
// Self-test of the bounded grid barrier: a cooperative launch whose barrier
// expects one CTA more than it has, so every wait must run out.  Returns
// GSI_ETIMEOUT when the kernel reported that, GSI_OK otherwise.
gsi_status selftest_barrier_timeout(int dev, unsigned long long spin_limit, double *ms);
// Seed + every join step of one query in one cooperative launch, in two
// parts.  query_coop_configs writes the k step configurations
// (join_args_size() * k bytes) to cfg_host and returns the dynamic shared
// memory the launch needs; the caller uploads them to cfg_dev together with
// the k step records (host-initialised static fields) and the zeroed control
// words.  launch_query_coop then launches; bsum: QUERY_MAX_CTAS words.
// steps[0].count receives |seed|.
// memo: query_memo_tables(steps, k) tables of n 8-byte entries, zeroed before
// the launch (per-vertex label sub-list locations, see join_rows.cuh), or null.
int query_memo_tables(const std::vector<JoinStep> &steps, int k);
gsi_status query_coop_configs(const gsi_graph *g, const std::vector<JoinStep> &steps, int k, const uint32_t *bitmaps,
                              const int32_t *order, int count_only, unsigned long long *stats, uint64_t *memo, bool nodedup,
                              void *cfg_host, size_t *smem);
// nodedup (configs): rows of single-edge steps are joined one by one (no
// warp groups, no memo).  listwise (launch): the kernel variant that also
// counts whole-list bytes (stats[2]).
gsi_status launch_query_coop(const gsi_graph *g, int k, const uint32_t *seed_bitmap, size_t smem, void *cfg_dev,
                             DStep *dsteps, QueryCtl *ctl, unsigned long long *bsum, int *grid_out, bool listwise,
                             cudaStream_t stream);

}  // namespace gsi

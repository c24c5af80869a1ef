// The candidate-slot tile of a join step, shared by the host-sized launch,
// the one-launch-per-query kernel and the batched kernel.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace gsi {

// [lo, hi) of the entries with label rank `r` inside the (rank, id)-sorted list cl[a..b)
__device__ inline void label_range(const uint16_t *__restrict__ cl, uint32_t a, uint32_t b, uint32_t r,
                                   uint32_t *lo, uint32_t *hi) {
    // the two bounds searched in lockstep: each round issues both probes,
    // so the chain of dependent loads is as long as one search
    uint32_t l1 = a, h1 = b, l2 = a, h2 = b;
    while (l1 < h1 || l2 < h2) {
        const uint32_t m1 = (l1 + h1) >> 1, m2 = (l2 + h2) >> 1;
        const uint32_t c1 = l1 < h1 ? __ldg(cl + m1) : 0u;
        const uint32_t c2 = l2 < h2 ? __ldg(cl + m2) : 0u;
        if (l1 < h1) {
            if (c1 < r) l1 = m1 + 1;
            else h1 = m1;
        }
        if (l2 < h2) {
            if (c2 <= r) l2 = m2 + 1;
            else h2 = m2;
        }
    }
    *lo = l1;
    *hi = l2;
}

struct StepDev {
    int32_t t, d, L, ulab;
    int32_t hom;                // 1: no set subtraction (homomorphism, Sec. VII-A)
    uint32_t inj;               // columns the set subtraction tests: those whose query vertex
                                // carries u's label (no other column can hold w); 0 under hom
    int32_t col[GSI_MAX_QUERY_VERTICES];
    int32_t lab[GSI_MAX_QUERY_VERTICES];
};

// Row i's output bound: the shortest label sub-list over its linking edges.
// `row` may have been written earlier in the same launch by other CTAs (the
// one-launch-per-query and batched kernels reuse their table regions), so it
// is read through L2 (ld.global.cg), never through the read-only path.
__device__ inline uint32_t row_bound(const StepDev &s, const int32_t *row, const uint32_t *__restrict__ off,
                                     const uint16_t *__restrict__ cl) {
    uint32_t best = 0xffffffffu;
    for (int j = 0; j < s.d; ++j) {
        uint64_t seg = (uint64_t)(uint32_t)__ldcg(row + s.col[j]) * (uint64_t)s.L + (uint64_t)s.lab[j];
        uint32_t a = __ldg(off + seg), b = __ldg(off + seg + 1), lo, hi;
        label_range(cl, a, b, (uint32_t)s.ulab, &lo, &hi);
        best = min(best, hi - lo);
        if (best == 0) break;
    }
    return best;
}

// Bits of a per-row bound record: the shortest sub-list's length in the low
// 27 bits, the index of its linking edge above (lists stay below 2^27).
constexpr uint32_t BOUND_LEN_BITS = 27;
constexpr uint32_t BOUND_LEN_MASK = (1u << BOUND_LEN_BITS) - 1;

// row_bound plus where the shortest sub-list starts and which linking edge
// gives it (the join tile then stages the row without searching again), and
// the summed length of all sub-lists.
__device__ inline uint32_t row_bound_full(const StepDev &s, const int32_t *row, const uint32_t *__restrict__ off,
                                          const uint16_t *__restrict__ cl, uint32_t *lo_best, int *jb,
                                          uint64_t *lsum) {
    uint32_t best = 0xffffffffu, bl = 0;
    int bj = 0;
    uint64_t sum = 0;
    for (int j = 0; j < s.d; ++j) {
        uint64_t seg = (uint64_t)(uint32_t)__ldcg(row + s.col[j]) * (uint64_t)s.L + (uint64_t)s.lab[j];
        uint32_t a = __ldg(off + seg), b = __ldg(off + seg + 1), lo, hi;
        label_range(cl, a, b, (uint32_t)s.ulab, &lo, &hi);
        if (hi - lo < best) {
            best = hi - lo;
            bl = lo;
            bj = j;
        }
        sum += hi - lo;
    }
    *lo_best = bl;
    *jb = bj;
    *lsum = sum;
    return best;
}

// Membership of x (label rank r) in a whole list ci[a..b), sorted by
// (label rank, id): binary search on the pair.
__device__ inline bool ranked_contains(const int32_t *__restrict__ ci, const uint16_t *__restrict__ cl, uint32_t a,
                                       uint32_t b, uint32_t r, int32_t x) {
    uint32_t lo = a, hi = b;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t cm = __ldg(cl + mid);
        const bool less = cm < r || (cm == r && __ldg(ci + mid) < x);
        if (less) lo = mid + 1;
        else hi = mid;
    }
    return lo < b && __ldg(cl + lo) == r && __ldg(ci + lo) == x;
}

// Algorithmic bytes of one row of a join step (t columns, d linking lists,
// label sub-lists summing to lsum, the shortest of length best): read the
// row, locate each list and its label sub-range, read the other sub-lists,
// and one list element plus one bitmap word per candidate slot.  Survivors
// add 4(t+1) each when written.
__device__ __forceinline__ unsigned long long row_alg_bytes(int t, int d, uint64_t lsum, uint32_t best) {
    return 4ull * t + 16ull * d + 4ull * (lsum - best) + 8ull * best;
}

// The same row under the whole-list model: read the row, locate each linking
// list with one 8-byte offset pair, read every linking list N(v, l) whole
// (wsum elements, the merge-intersection bound), and probe the bitmap once
// per candidate slot.  Survivors add 4(t+1) each, as above.
__device__ __forceinline__ unsigned long long row_list_bytes(int t, int d, uint64_t wsum, uint32_t best) {
    return 4ull * t + 8ull * d + 4ull * wsum + 4ull * best;
}

struct JoinArgs {
    const int32_t *M;
    int64_t R;
    const uint64_t *F;
    uint64_t total;
    const int64_t *part;
    const uint32_t *off;
    const int32_t *ci;
    const uint16_t *cl;
    const uint32_t *cand;
    int32_t *out;
    uint64_t out_cap;
    unsigned long long *out_count;
    unsigned long long *stats;
    int32_t W, rmax, count_only;
    StepDev s;
    int32_t iperm[GSI_MAX_QUERY_VERTICES + 1];   // output column oc holds input position iperm[oc]
    // per-vertex memo of label sub-list locations for the first linking edges
    // (null: none); table j holds n entries, tagged with the step
    uint64_t *memo;
    int64_t memo_n;
    int32_t isect;              // intersection strategy of short multi-edge rows (ISECT_*)
    int32_t nodedup;            // 1: no duplicate removal in the row pass (no warp groups, no memo)
};

// How a short row's candidates are intersected with its other linking lists
// (all give the same set; the batched autotuner picks one per batch):
//   ISECT_BSEARCH  each candidate is searched in each other label sub-list;
//   ISECT_MERGE    each other sub-list is walked once beside the candidates
//                  (both ascending), a two-pointer merge;
//   ISECT_BITMAP   each element of each other sub-list is searched among the
//                  candidates, setting a bit per candidate position; the
//                  masks of all lists are ANDed.
constexpr int ISECT_BSEARCH = 0, ISECT_MERGE = 1, ISECT_BITMAP = 2;

template <int NT>
__device__ inline int block_inclusive_max(int v, int *wt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= o) v = max(v, y);
    }
    if (lane == 31) wt[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? wt[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL_MASK, w, o);
            if (lane >= o) w = max(w, y);
        }
        if (lane < NW) wt[lane] = w;
    }
    __syncthreads();
    int r = warp > 0 ? max(v, wt[warp - 1]) : v;
    __syncthreads();
    return r;
}

constexpr int MEMO_EDGES = 4;     // linking edges of a step with a sub-list memo
constexpr uint32_t MEMO_TAG_SHIFT = 59;

// Start (*lo) and length (returned) of the label(u) sub-list of N(v, lab[j]),
// through the memo when the step has one.  A memo entry is
// start | length << 32 | step << MEMO_TAG_SHIFT; concurrent writers store the
// same value, and a load that sees an older entry (another step's, or a
// stale cached line) only recomputes it.
__device__ __forceinline__ uint32_t sublist(const JoinArgs &a, int j, int32_t v, uint32_t *lo) {
    uint64_t *slot = nullptr;
    uint64_t e = 0;
    const uint64_t seg = (uint64_t)(uint32_t)v * (uint64_t)a.s.L + (uint64_t)a.s.lab[j];
    if (a.memo && j < MEMO_EDGES) {
        slot = a.memo + (uint64_t)j * (uint64_t)a.memo_n + (uint32_t)v;
        e = *slot;
    }
    // the list's offsets are loaded beside the memo entry (used on a miss)
    const uint32_t x0 = __ldg(a.off + seg), x1 = __ldg(a.off + seg + 1);
    if (slot && (uint32_t)(e >> MEMO_TAG_SHIFT) == (uint32_t)a.s.t) {
        *lo = (uint32_t)e;
        return (uint32_t)(e >> 32) & BOUND_LEN_MASK;
    }
    uint32_t l, h;
    label_range(a.cl, x0, x1, (uint32_t)a.s.ulab, &l, &h);
    *lo = l;
    const uint32_t len = h - l;
    if (slot && len <= BOUND_LEN_MASK)
        *slot = (uint64_t)l | ((uint64_t)len << 32) | ((uint64_t)(uint32_t)a.s.t << MEMO_TAG_SHIFT);
    return len;
}

// One tile of NV candidate slots.  The table-dependent inputs (M, R, F,
// total, part, out, out_cap, out_count) are arguments so that the same code
// serves host-sized launches (one CTA per tile) and device-sized persistent
// launches (CTAs take tiles from a counter).  M and F can be rewritten within
// one persistent launch (ping-pong table regions, one scratch region for
// every step), so they are read through L2 (ld.global.cg) and never through
// the non-coherent read-only path.
//
// With bounds (PRE: the long rows set aside by the row pass), each row's
// shortest label sub-list is already known: bnd[r] holds its length and
// linking-edge index (BOUND_LEN_BITS), blo[r] its start.  Staging then reads
// those instead of searching, the other linking lists' label(u) sub-lists
// come from the step's memo (filled by the row pass) or a label-range search,
// and since every such row spans more than
// SHORT_MAX + W slots a tile holds few rows, so each slot finds its row by a
// binary search of the staged offsets instead of a block-wide scan.
template <int NT, int VT, bool TILE_STATS = true, bool PRE = false>
__device__ __forceinline__ void join_tile(const JoinArgs &a, const int32_t *M, int64_t R,
                                          const uint64_t *F, uint64_t total, int64_t r_lo,
                                          int64_t r_next, int32_t *__restrict__ out, uint64_t out_cap,
                                          unsigned long long *out_count, uint64_t tile,
                                          const uint32_t *bnd = nullptr, const uint32_t *blo = nullptr) {
    constexpr int NV = NT * VT;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long wt[NT / 32];
    __shared__ int wti[NT / 32];
    __shared__ unsigned long long gbase_s;
    __shared__ unsigned wcnt[NT / 32 + 1];

    const int t = a.s.t, d = a.s.d, dm1 = d - 1;
    // dynamic shared memory (join_smem): per-warp survivors (local row, w),
    // row offsets, candidate sub-list starts, other lists, staged rows, and
    // the slot -> row map
    int2 (*wsurv)[32 * VT] = reinterpret_cast<int2 (*)[32 * VT]>(smem);  // NT / 32 warps
    uint64_t *Fs = reinterpret_cast<uint64_t *>(smem + (size_t)NV * 8);  // rmax + 1
    uint32_t *base0 = reinterpret_cast<uint32_t *>(Fs + a.rmax + 1);    // rmax
    uint32_t *lst = base0 + a.rmax;                                     // rmax * 2 * dm1
    int32_t *rowv = reinterpret_cast<int32_t *>(lst + (size_t)a.rmax * 2 * dm1);   // rmax * t
    uint16_t *rowmap = reinterpret_cast<uint16_t *>(rowv + (size_t)a.rmax * t);   // NV

    // rows r_lo .. min(r_next, R-1): r_lo holds slot s0, r_next holds slot s0 + NV
    const uint64_t s0 = tile * NV;
    const uint64_t s1 = min(s0 + (uint64_t)NV, total);
    const int64_t r_hi = min(r_next, R - 1);
    const int nr = (int)(r_hi - r_lo + 1);

    // ---- stage the tile's rows: values, candidate sub-list, other sub-lists
    if (!PRE)
        for (int x = threadIdx.x; x < NV; x += NT) rowmap[x] = 0;
    for (int lr = threadIdx.x; lr <= nr; lr += NT) Fs[lr] = __ldcg(F + r_lo + lr);
    __syncthreads();
    unsigned long long bytes = 0;
    for (int lr = threadIdx.x; lr < nr; lr += NT) {
        const int32_t *row = M + (r_lo + lr) * (int64_t)t;
        int32_t *rv = rowv + lr * t;
        for (int c = 0; c < t; ++c) rv[c] = __ldcg(row + c);
        if (PRE) {
            // the bound scan's record: candidates from the shortest sub-list;
            // every other linking list restricted to label(u)
            const uint32_t bw = __ldcg(bnd + r_lo + lr);
            const uint32_t best = bw & BOUND_LEN_MASK;
            const int jb = (int)(bw >> BOUND_LEN_BITS);
            base0[lr] = __ldcg(blo + r_lo + lr);
            int q = 0;
            for (int j = 0; j < d && best > 0; ++j) {
                if (j == jb) continue;
                uint32_t lo;
                const uint32_t len = sublist(a, j, rv[a.s.col[j]], &lo);
                lst[(lr * dm1 + q) * 2] = lo;
                lst[(lr * dm1 + q) * 2 + 1] = len;
                ++q;
            }
            continue;
        }
        // the row's lists: the shortest label sub-list supplies candidates
        uint32_t lo[GSI_MAX_QUERY_VERTICES], len[GSI_MAX_QUERY_VERTICES];
        uint32_t best = 0xffffffffu;
        int jb = 0;
        uint64_t lsum = 0;
        for (int j = 0; j < d; ++j) {
            uint64_t seg = (uint64_t)(uint32_t)rv[a.s.col[j]] * (uint64_t)a.s.L + (uint64_t)a.s.lab[j];
            uint32_t x0 = __ldg(a.off + seg), x1 = __ldg(a.off + seg + 1), h;
            label_range(a.cl, x0, x1, (uint32_t)a.s.ulab, &lo[j], &h);
            len[j] = h - lo[j];
            if (len[j] < best) { best = len[j]; jb = j; }
            lsum += len[j];
            if (best == 0) break;
        }
        base0[lr] = lo[jb];
        int q = 0;
        for (int j = 0; j < d && best > 0; ++j) {
            if (j == jb) continue;
            lst[(lr * dm1 + q) * 2] = lo[j];
            lst[(lr * dm1 + q) * 2 + 1] = len[j];
            ++q;
        }
        const uint64_t fr = Fs[lr];
        if (fr > s0 && fr < s1) rowmap[fr - s0] = (uint16_t)lr;       // first slot of the row in this tile
        if (TILE_STATS && a.stats && fr >= s0) bytes += 4ull * t + 8ull * d + 4ull * (lsum - best);   // row owned by this tile
    }
    __syncthreads();
    if (!PRE) {   // slot -> row: inclusive max-scan of the row-start marks
        int v[VT];
        int m = 0;
#pragma unroll
        for (int k = 0; k < VT; ++k) {
            v[k] = rowmap[threadIdx.x * VT + k];
            m = max(m, v[k]);
            v[k] = m;
        }
        const int incl = block_inclusive_max<NT>(m, wti);   // max over threads 0..tid
        const int before = __shfl_up_sync(FULL_MASK, incl, 1);
        // exclusive prefix for this thread = inclusive max of the previous thread
        int ex = 0;
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (lane > 0) ex = before;
            else if (warp > 0) ex = wti[warp - 1];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < VT; ++k) rowmap[threadIdx.x * VT + k] = (uint16_t)max(ex, v[k]);
        __syncthreads();
    }

    // ---- candidates: one slot per thread per round, consecutive slots per
    // warp; the VT slots' list loads, then their bitmap probes, are issued
    // together
    int32_t wv[VT];
    int32_t lrv[VT];
    uint32_t cix[VT];
    unsigned okmask = 0, vmask = 0;
    unsigned long long items = 0;
#pragma unroll
    for (int k = 0; k < VT; ++k) {
        const uint64_t s = s0 + (uint64_t)(k * NT + threadIdx.x);
        wv[k] = 0;
        lrv[k] = 0;
        cix[k] = 0;
        if (s >= s1) continue;
        int lr;
        if (PRE) {
            // long rows only (each holds more than SHORT_MAX + W slots): few
            // rows per tile, found by a search of the staged offsets
            int l = 0, h = nr - 1;
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (Fs[mid] <= s) l = mid;
                else h = mid - 1;
            }
            lr = l;
        } else {
            lr = rowmap[s - s0];
        }
        const int64_t p = (int64_t)(s - Fs[lr]) - a.W;
        lrv[k] = lr;
        if (p < 0) continue;            // a row-staging slot
        ++items;
        cix[k] = base0[lr] + (uint32_t)p;
        vmask |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < VT; ++k)
        if ((vmask >> k) & 1u) wv[k] = __ldg(a.ci + cix[k]);
    uint32_t bw[VT];
#pragma unroll
    for (int k = 0; k < VT; ++k) bw[k] = ((vmask >> k) & 1u) ? __ldg(a.cand + (wv[k] >> 5)) : 0u;
#pragma unroll
    for (int k = 0; k < VT; ++k) {
        const int32_t w = wv[k];
        bool ok = (bw[k] >> (w & 31)) & 1u;
        const int32_t *rv = rowv + lrv[k] * t;
        for (uint32_t im = a.s.inj; ok && im; im &= im - 1) ok = rv[__ffs(im) - 1] != w;
        for (int j = 0; j < dm1 && ok; ++j) {
            const uint32_t *ls = lst + (lrv[k] * dm1 + j) * 2;
            ok = sorted_contains(a.ci + ls[0], ls[1], w);
        }
        if (ok) okmask |= 1u << k;
    }

    // ---- compaction: warp ballots, one atomic per CTA, then each warp writes
    // its survivors' rows as one contiguous, coalesced run of M'
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned nw = 0;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < VT; ++k) {
        const bool ok = (okmask >> k) & 1u;
        const unsigned b = __ballot_sync(FULL_MASK, ok);
        if (ok) wsurv[warp][nw + __popc(b & lt)] = make_int2(lrv[k], wv[k]);
        nw += __popc(b);
    }
    if (lane == 0) wcnt[warp] = nw;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int w = 0; w < NT / 32; ++w) {
            unsigned c = wcnt[w];
            wcnt[w] = run;
            run += c;
        }
        wcnt[NT / 32] = run;
        gbase_s = run ? atomicAdd(out_count, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    const unsigned nsurv = wcnt[NT / 32];
    if (!a.count_only && nw > 0) {
        const uint64_t base = gbase_s + wcnt[warp];
        const uint64_t room = out_cap > base ? out_cap - base : 0;
        const unsigned nrow = (unsigned)min((uint64_t)nw, room);
        // fixed lane map: lane = rs * W1 + oc writes column oc of the rs-th of
        // rpw rows per round, so each round stores one contiguous run
        const int W1 = t + 1;
        const int rpw = 32 / W1, rs = lane / W1, oc = lane - rs * W1;
        const int c = a.iperm[oc];
        int32_t *dst = out + base * (uint64_t)W1;
        if (rs < rpw)
            for (unsigned r = (unsigned)rs; r < nrow; r += (unsigned)rpw) {
                const int2 sv = wsurv[warp][r];
                dst[(uint64_t)r * W1 + oc] = c == t ? sv.y : rowv[sv.x * t + c];
            }
    }
    if (TILE_STATS && a.stats) {
        bytes += 8ull * items;                                    // list element + bitmap probe
        if (!a.count_only && threadIdx.x == 0) bytes += 4ull * (t + 1) * nsurv;
        unsigned long long bsum = block_sum<NT, unsigned long long>(bytes, wt);
        unsigned long long isum = block_sum<NT, unsigned long long>(items, wt);
        if (threadIdx.x == 0) {
            atomicAdd(a.stats, bsum);
            atomicAdd(a.stats + 1, isum);
        }
    }
}

// Dynamic shared memory of join_tile for rmax staged rows of t columns and d lists.
size_t join_smem(int rmax, int t, int d);
// Static configuration of one join step (candidate bitmap, lists, permutation).
JoinArgs make_join_args(const gsi_graph *g, const JoinStep &s, const uint32_t *cand, int count_only,
                        unsigned long long *stats);

}  // namespace gsi

// The row pass of a join step: short rows joined by one thread each, long
// rows set aside for the candidate-slot tiles.
//
// Most rows of the large steps have one or two candidates in their shortest
// label sub-list (the Alg. 4 bound).  For such a row the slot-tile path pays
// more for the bookkeeping (a bound record, a slot offset, a tile partition,
// staging, a slot-to-row map and W staging slots) than for the join itself.
// Here one thread takes one row from its bound to its survivors in a single
// pass:
//   * a CTA stages NT consecutive rows of M with coalesced loads;
//   * each thread finds its row's shortest label sub-list over the linking
//     edges (the output bound, Alg. 4);
//   * when that bound is at most SHORT_MAX, the thread tests every candidate
//     (bitmap of C(u), set subtraction against the row, membership in the
//     other linking lists: Alg. 3's set operations) and keeps a bit mask of
//     survivors;
//   * otherwise the row, with its bound record (length, linking edge, start),
//     is appended to a long-row table that the slot tiles process after a
//     grid barrier (a hub row then spreads over many CTAs, Sec. VI-A's load
//     balancing done by the tiles);
//   * one block-wide scan and one atomic per CTA and batch place the batch's
//     survivors in M', which the CTA writes as one coalesced run
//     (Prealloc-Combine without a second join: each survivor is written
//     once).
//
// Shared work between rows (duplicate removal, Sec. VI-B).  Rows of a step
// reuse few data vertices: consecutive rows of M' often extend the same
// row of M, and hubs recur everywhere.  Two mechanisms keep rows from
// repeating each other's work:
//   * a per-step memo holds, for each data vertex v and each of the first
//     MEMO_EDGES linking edges, where the label(u) sub-list of N(v, l) starts
//     and how long it is; a row whose vertex is in the memo skips the list
//     lookup and the label-range search (entries carry the step number, so a
//     stale entry is a miss, never a wrong answer);
//   * in single-edge steps the lanes of a warp whose rows share the first-edge
//     vertex v (found with __match_any_sync) elect one lane, which locates the
//     sub-list and probes the candidate bitmap C(u) for the whole group once;
//     the other lanes receive the bound and the bitmap mask by shuffle and
//     only add their own set subtraction, as Alg. 5 shares one N(v, l0)
//     fetch among the rows of a block that have the same m_i[u0'].
#pragma once

#include "join_tile.cuh"

namespace gsi {

constexpr int SHORT_MAX = 16;     // rows with at most this many candidates are joined inline
// Rows of one slot tile of long rows: every long row spans at least
// SHORT_MAX + 1 + W slots, plus a partial row at each end of the tile.
constexpr int LONG_RMAX = JOIN_NV / (SHORT_MAX + 1 + JOIN_ROW_WEIGHT) + 2;

// Rows whose bound exceeds SHORT_MAX, copied (t columns) with their bound
// records, for the slot tiles.  count is a device counter.
struct LongTable {
    int32_t *rows;
    uint32_t *bnd;                // length | linking edge << BOUND_LEN_BITS
    uint32_t *blo;                // start of the shortest sub-list
    uint64_t cap;                 // rows the table holds
    unsigned long long *count;
};

// Layout of the long-row table of step t in a scratch region of S_words
// 8-byte words: rows, bound records, then F; the tile partition takes what is
// left (at least an eighth of the region).
struct LongLayout {
    uint64_t cap, f_off, part_off, part_cap;    // offsets in words
};
__host__ __device__ inline LongLayout long_layout(uint64_t S_words, int t) {
    LongLayout l;
    const uint64_t avail = S_words > 64 ? S_words - S_words / 8 - 8 : 0;
    l.cap = avail * 8 / (4ull * (uint64_t)t + 16ull);
    const uint64_t rec_words = (l.cap * (4ull * (uint64_t)t + 8ull) + 7) / 8;
    l.f_off = rec_words;
    l.part_off = l.f_off + l.cap + 1;
    l.part_cap = S_words > l.part_off ? S_words - l.part_off : 0;
    return l;
}

constexpr int ROW_RPT = 2;        // rows per thread in one batch of the row pass
constexpr int ROW_SURV = 4;       // survivor-list entries per batch row (more are written in rounds)

// Dynamic shared memory of the row pass for CTAs of nt threads: nt * ROW_RPT
// staged rows of t columns, their candidate sub-list starts, then the
// survivor list (values, local row and candidate position).
__host__ __device__ constexpr size_t rows_smem(int nt, int t, int rpt = ROW_RPT) {
    return (size_t)nt * rpt * ((size_t)t * 4 + 4) + (size_t)nt * rpt * ROW_SURV * 6;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA engine, no registers or
// shared memory involved): the start is rounded up and the size down to 16
// bytes, so the prefetch never reaches past the range.
__device__ __forceinline__ void prefetch_l2(const void *p, uint64_t bytes) {
    const uint64_t a = (uint64_t)reinterpret_cast<uintptr_t>(p);
    const uint64_t end = (a + bytes) & ~15ull;
    for (uint64_t x = (a + 15) & ~15ull; x < end;) {
        const uint32_t chunk = (uint32_t)min(end - x, (uint64_t)1 << 20);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(x), "r"(chunk) : "memory");
        x += chunk;
    }
}

// Copies n int32 from global src to shared dst (16-byte aligned) through L2
// (the rows may have been written by other SMs), spread over NT threads: in
// 16-byte pieces when src is 16-byte aligned, four pieces in flight per
// thread; element by element otherwise.
template <int NT>
__device__ __forceinline__ void stage_rows(int32_t *dst, const int32_t *__restrict__ src, int n) {
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int nv = n >> 2;
        const int4 *s4 = reinterpret_cast<const int4 *>(src);
        int4 *d4 = reinterpret_cast<int4 *>(dst);
        int i = threadIdx.x;
        for (; i + 3 * NT < nv; i += 4 * NT) {
            const int4 x0 = __ldcg(s4 + i), x1 = __ldcg(s4 + i + NT), x2 = __ldcg(s4 + i + 2 * NT),
                       x3 = __ldcg(s4 + i + 3 * NT);
            d4[i] = x0;
            d4[i + NT] = x1;
            d4[i + 2 * NT] = x2;
            d4[i + 3 * NT] = x3;
        }
        for (; i < nv; i += NT) d4[i] = __ldcg(s4 + i);
        for (int e = nv * 4 + threadIdx.x; e < n; e += NT) dst[e] = __ldcg(src + e);
    } else {
        for (int e = threadIdx.x; e < n; e += NT) dst[e] = __ldcg(src + e);
    }
}

// Length of the whole linking list N(v, lab[j]) (for the whole-list byte count).
__device__ __forceinline__ uint32_t whole_len(const JoinArgs &a, int j, int32_t v) {
    const uint64_t seg = (uint64_t)(uint32_t)v * (uint64_t)a.s.L + (uint64_t)a.s.lab[j];
    return __ldg(a.off + seg + 1) - __ldg(a.off + seg);
}

// Candidates ci[lo + p], p < len <= 32, that are in C(u): bit p of the result.
__device__ __forceinline__ uint32_t bitmap_mask(const JoinArgs &a, uint32_t lo, uint32_t len) {
    uint32_t mask = 0;
    for (uint32_t p0 = 0; p0 < len; p0 += 4) {
        int32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = p0 + q < len ? __ldg(a.ci + lo + p0 + q) : -1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (w[q] >= 0 && ((__ldg(a.cand + (w[q] >> 5)) >> (w[q] & 31)) & 1u)) mask |= 1u << (p0 + q);
    }
    return mask;
}

// Clears the bits of `mask` whose candidate equals a value of the row in a
// column the set subtraction tests (only columns whose query vertex carries
// u's label can hold w; none under homomorphism).
__device__ __forceinline__ uint32_t subtract_row(const JoinArgs &a, const int32_t *row, uint32_t lo, uint32_t mask) {
    const uint32_t inj = a.s.inj;
    if (!inj) return mask;
    for (uint32_t m = mask; m; m &= m - 1) {
        const int p = __ffs(m) - 1;
        const int32_t w = __ldg(a.ci + lo + (uint32_t)p);
        for (uint32_t im = inj; im; im &= im - 1)
            if (row[__ffs(im) - 1] == w) {
                mask &= ~(1u << p);
                break;
            }
    }
    return mask;
}

// One row of the pass: its bound (shortest label sub-list: length *best,
// start *lob, linking edge *jb) and the mask of its survivors among the
// first *best candidates when best <= SHORT_MAX.  Lanes whose rows share the
// first-edge vertex of a single-edge step share the lookup and the bitmap
// probes (every lane of the warp must call this together).
template <bool DR, bool LW = true>
__device__ __forceinline__ uint32_t row_join(const JoinArgs &a, const int32_t *row, bool valid, int lane,
                                             uint32_t *best_out, uint32_t *lob_out, int *jb_out,
                                             unsigned long long *abytes, unsigned long long *items,
                                             unsigned long long *lbytes) {
    const int t = a.s.t, d = a.s.d;
    const bool stats = a.stats != nullptr;
    uint32_t mask = 0, best = 0, lob = 0;
    int jb = 0;
    if (DR && d == 1) {
        const int32_t v = valid ? row[a.s.col[0]] : -1 - lane;
        const unsigned peers = __match_any_sync(FULL_MASK, v);
        const int leader = __ffs(peers) - 1;
        uint32_t bm = 0;
        if (lane == leader && valid) {
            best = sublist(a, 0, v, &lob);
            if (best <= (uint32_t)SHORT_MAX) bm = bitmap_mask(a, lob, best);
        }
        best = __shfl_sync(FULL_MASK, best, leader);
        lob = __shfl_sync(FULL_MASK, lob, leader);
        bm = __shfl_sync(FULL_MASK, bm, leader);
        if (valid && best <= (uint32_t)SHORT_MAX) mask = subtract_row(a, row, lob, bm);
        if (valid && stats) {
            *abytes += row_alg_bytes(t, 1, best, best);
            if (LW) *lbytes += row_list_bytes(t, 1, whole_len(a, 0, v), best);
            *items += best;
        }
    } else if (valid) {
        uint32_t lo4[MEMO_EDGES], len4[MEMO_EDGES];
        uint64_t lsum = 0;
        best = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < MEMO_EDGES; ++j) {
            lo4[j] = 0;
            len4[j] = 0;
            if (j < d) {
                len4[j] = sublist(a, j, row[a.s.col[j]], &lo4[j]);
                lsum += len4[j];
                if (len4[j] < best) {
                    best = len4[j];
                    lob = lo4[j];
                    jb = j;
                }
            }
        }
        for (int j = MEMO_EDGES; j < d; ++j) {
            uint32_t l;
            const uint32_t n = sublist(a, j, row[a.s.col[j]], &l);
            lsum += n;
            if (n < best) {
                best = n;
                lob = l;
                jb = j;
            }
        }
        if (stats) {
            if (LW) {
                uint64_t wsum = 0;
                for (int j = 0; j < d; ++j) wsum += whole_len(a, j, row[a.s.col[j]]);
                *lbytes += row_list_bytes(t, d, wsum, best);
            }
            *abytes += row_alg_bytes(t, d, lsum, best);
            *items += best;
        }
        if (best > 0 && best <= (uint32_t)SHORT_MAX) {
            mask = subtract_row(a, row, lob, bitmap_mask(a, lob, best));
            // every other linking list must hold the candidate (Alg. 3)
            if (a.isect == ISECT_BSEARCH) {
                for (uint32_t m = mask; m; m &= m - 1) {
                    const int p = __ffs(m) - 1;
                    const int32_t w = __ldg(a.ci + lob + (uint32_t)p);
                    bool ok = true;
#pragma unroll
                    for (int j = 0; j < MEMO_EDGES; ++j)
                        if (ok && j < d && j != jb) ok = sorted_contains(a.ci + lo4[j], len4[j], w);
                    if (!ok) mask &= ~(1u << p);
                }
            } else {
#pragma unroll
                for (int j = 0; j < MEMO_EDGES; ++j) {
                    if (!mask || j >= d || j == jb) continue;
                    uint32_t keep = 0;
                    const uint32_t b0 = lo4[j], b1 = lo4[j] + len4[j];
                    if (a.isect == ISECT_MERGE) {
                        // both lists ascend: one pointer into the other list
                        uint32_t q = b0;
                        for (uint32_t m = mask; m && q < b1; m &= m - 1) {
                            const int p = __ffs(m) - 1;
                            const int32_t w = __ldg(a.ci + lob + (uint32_t)p);
                            while (q < b1 && __ldg(a.ci + q) < w) ++q;
                            if (q < b1 && __ldg(a.ci + q) == w) keep |= 1u << p;
                        }
                    } else {
                        // every element of the other list marks its position
                        // among the candidates
                        for (uint32_t q = b0; q < b1; ++q) {
                            const int32_t x = __ldg(a.ci + q);
                            uint32_t l = 0, h = best;
                            while (l < h) {
                                const uint32_t mid = (l + h) >> 1;
                                if (__ldg(a.ci + lob + mid) < x) l = mid + 1;
                                else h = mid;
                            }
                            if (l < best && __ldg(a.ci + lob + l) == x) keep |= 1u << l;
                        }
                    }
                    mask &= keep;
                }
            }
            for (int j = MEMO_EDGES; j < d && mask; ++j) {      // lists without a memo slot: searched whole
                if (j == jb) continue;
                const uint64_t seg = (uint64_t)(uint32_t)row[a.s.col[j]] * (uint64_t)a.s.L + (uint64_t)a.s.lab[j];
                const uint32_t x0 = __ldg(a.off + seg), x1 = __ldg(a.off + seg + 1);
                for (uint32_t m = mask; m; m &= m - 1) {
                    const int p = __ffs(m) - 1;
                    if (!ranked_contains(a.ci, a.cl, x0, x1, (uint32_t)a.s.ulab, __ldg(a.ci + lob + (uint32_t)p)))
                        mask &= ~(1u << p);
                }
            }
        }
    }
    *best_out = best;
    *lob_out = lob;
    *jb_out = jb;
    return mask;
}

// The single-edge rows of one thread (RPT of them, rows q * NT + tid) in
// lockstep, so that each round of loads is issued for all of them at once:
// first-edge vertices and their warp groups, memo lookups (the leader of each
// group), candidate values, bitmap probes, then the group's bound and bitmap
// mask to every lane, and each lane's own set subtraction.  Sets best[q],
// lob[q] and mask[q]; rows past nb get best 0.
constexpr int ROW_C = 8;          // candidate values of a single-edge group loaded in the first round

template <int NT, int RPT, bool LW = true>
__device__ __forceinline__ void rows_join_single(const JoinArgs &a, const int32_t *rowv, int nb, int lane,
                                                 uint32_t *best, uint32_t *lob, uint32_t *mask,
                                                 unsigned long long *abytes, unsigned long long *items,
                                                 unsigned long long *lbytes) {
    constexpr int C = ROW_C;
    const int t = a.s.t;
    int32_t v[RPT];
    bool lead[RPT];
    int leader[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int lr = q * NT + (int)threadIdx.x;
        v[q] = lr < nb ? rowv[lr * t + a.s.col[0]] : -1 - lane;
        const unsigned peers = __match_any_sync(FULL_MASK, v[q]);
        leader[q] = __ffs(peers) - 1;
        lead[q] = lane == leader[q] && lr < nb;
    }
    // memo lookups of the group leaders, with the list offsets beside them
    // (used on a miss)
    uint64_t e[RPT];
    uint32_t x0[RPT], x1[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        e[q] = (lead[q] && a.memo) ? a.memo[(uint32_t)v[q]] : 0ull;
        const uint64_t seg = (uint64_t)(uint32_t)(lead[q] ? v[q] : 0) * (uint64_t)a.s.L + (uint64_t)a.s.lab[0];
        x0[q] = lead[q] ? __ldg(a.off + seg) : 0u;
        x1[q] = lead[q] ? __ldg(a.off + seg + 1) : 0u;
    }
    uint32_t len[RPT], lo[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        len[q] = 0;
        lo[q] = 0;
        if (!lead[q]) continue;
        if (a.memo && (uint32_t)(e[q] >> MEMO_TAG_SHIFT) == (uint32_t)a.s.t) {
            lo[q] = (uint32_t)e[q];
            len[q] = (uint32_t)(e[q] >> 32) & BOUND_LEN_MASK;
        } else {
            uint32_t h;
            label_range(a.cl, x0[q], x1[q], (uint32_t)a.s.ulab, &lo[q], &h);
            len[q] = h - lo[q];
            if (a.memo && len[q] <= BOUND_LEN_MASK)
                a.memo[(uint32_t)v[q]] = (uint64_t)lo[q] | ((uint64_t)len[q] << 32) |
                                         ((uint64_t)(uint32_t)a.s.t << MEMO_TAG_SHIFT);
        }
    }
    // the first C candidates of every short group, then their bitmap probes
    int32_t w[RPT][C];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int p = 0; p < C; ++p)
            w[q][p] = (lead[q] && (uint32_t)p < len[q] && len[q] <= (uint32_t)SHORT_MAX)
                          ? __ldg(a.ci + lo[q] + (uint32_t)p) : -1;
    uint32_t bm[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        bm[q] = 0;
#pragma unroll
        for (int p = 0; p < C; ++p)
            if (w[q][p] >= 0 && ((__ldg(a.cand + (w[q][p] >> 5)) >> (w[q][p] & 31)) & 1u)) bm[q] |= 1u << p;
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q)                     // candidates past the first C (groups with C < len <= SHORT_MAX)
        if (lead[q] && len[q] > (uint32_t)C && len[q] <= (uint32_t)SHORT_MAX)
            bm[q] |= bitmap_mask(a, lo[q] + C, len[q] - C) << C;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int lr = q * NT + (int)threadIdx.x;
        const bool valid = lr < nb;
        best[q] = __shfl_sync(FULL_MASK, len[q], leader[q]);
        lob[q] = __shfl_sync(FULL_MASK, lo[q], leader[q]);
        const uint32_t b = __shfl_sync(FULL_MASK, bm[q], leader[q]);
        if (!valid) best[q] = 0;
        mask[q] = (valid && best[q] <= (uint32_t)SHORT_MAX) ? subtract_row(a, rowv + lr * t, lob[q], b) : 0u;
        if (a.stats) {
            if (LW) {                                 // whole first-edge list, from the group leader
                const uint32_t whole = __shfl_sync(FULL_MASK, lead[q] ? whole_len(a, 0, v[q]) : 0u, leader[q]);
                if (valid) *lbytes += row_list_bytes(t, 1, whole, best[q]);
            }
            if (valid) {
                *abytes += row_alg_bytes(t, 1, best[q], best[q]);
                *items += best[q];
            }
        }
    }
}

// The row pass over rows [first, R) in batches of NT * RPT rows, batch
// starts `stride` apart (a grid-strided pass: first = blockIdx.x * NB,
// stride = gridDim.x * NB; one CTA alone: first = 0, stride = NB).  `a` should
// live in shared memory.  Survivors go to out (up to cap rows; `count` is
// exact), long rows to lt.  Bit 1 of *fail is set when the long-row table is
// full or a bound does not fit its record.  When a.stats is set, adds this
// thread's algorithmic bytes (rows read, lists located and read; survivors
// are counted by the caller) to *abytes, the same under the whole-list model
// to *lbytes (only when LW), and its candidate slots to *items.
template <int NT, bool DR = true, int RPT = ROW_RPT, bool LW = true>
__device__ void row_pass(const JoinArgs &a, const int32_t *M, uint64_t R, uint64_t first, uint64_t stride,
                         int32_t *__restrict__ out, uint64_t cap, unsigned long long *count, const LongTable &lt,
                         unsigned *fail, unsigned char *smem, unsigned long long *abytes,
                         unsigned long long *items, unsigned long long *lbytes) {
    constexpr int NW = NT / 32, NB = NT * RPT, CCAP = NB * ROW_SURV;
    __shared__ uint32_t wt[NW];
    __shared__ unsigned long long base_s, lbase_s;
    const int t = a.s.t, W1 = t + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *rowv = reinterpret_cast<int32_t *>(smem);                  // NB * t
    uint32_t *lobs = reinterpret_cast<uint32_t *>(rowv + NB * t);        // NB
    int32_t *comp_w = reinterpret_cast<int32_t *>(lobs + NB);           // CCAP
    uint16_t *comp_r = reinterpret_cast<uint16_t *>(comp_w + CCAP);     // local row | position << 10
    const bool write = cap > 0;
    // the output loop's fixed lane map: lane = rs * W1 + c writes column c of
    // the rs-th of the warp's rpw rows per round
    const int rpw = 32 / W1, rs = lane / W1, oc = lane - rs * W1;
    const int src_col = a.iperm[oc < W1 ? oc : 0];
    for (uint64_t r0 = first; r0 < R; r0 += stride) {
        const int nb = (int)min((uint64_t)NB, R - r0);
        const int32_t *src = M + r0 * (uint64_t)t;
        if (threadIdx.x == 0 && r0 + stride < R)      // the next batch's rows, while this one runs
            prefetch_l2(M + (r0 + stride) * (uint64_t)t, min((uint64_t)NB, R - r0 - stride) * (uint64_t)t * 4);
        stage_rows<NT>(rowv, src, nb * t);
        __syncthreads();
        // this thread's rows q * NT + tid, q < RPT (a warp's lanes hold
        // consecutive rows)
        uint32_t mask[RPT], best[RPT], lob[RPT];
        int jb[RPT];
        uint32_t n = 0, nl = 0;
        if (DR && a.s.d == 1 && !a.nodedup) {
            rows_join_single<NT, RPT, LW>(a, rowv, nb, lane, best, lob, mask, abytes, items, lbytes);
#pragma unroll
            for (int q = 0; q < RPT; ++q) jb[q] = 0;
        } else {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int lr = q * NT + (int)threadIdx.x;
                const bool valid = lr < nb;
                mask[q] = row_join<false, LW>(a, rowv + (valid ? lr : 0) * t, valid, lane, &best[q], &lob[q], &jb[q],
                                          abytes, items, lbytes);
                if (!valid) best[q] = 0;
            }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            n += __popc(mask[q]);
            nl += best[q] > (uint32_t)SHORT_MAX;
        }
        // one barrier: warp scans, warp totals through shared memory (wt is
        // written again only after the next batch's staging barrier)
        uint32_t ex, tot;
        {
            const uint32_t v = n | (nl << 16);
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wt[warp] = x;
            __syncthreads();
            uint32_t pre = 0;
            tot = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t y = wt[w];
                pre += w < warp ? y : 0u;
                tot += y;
            }
            ex = pre + x - v;
        }
        const uint32_t ntot = tot & 0xffffu, ltot = tot >> 16;
        if (threadIdx.x == 0) {                 // read after the next barrier
            base_s = ntot ? atomicAdd(count, (unsigned long long)ntot) : 0ull;
            lbase_s = ltot ? atomicAdd(lt.count, (unsigned long long)ltot) : 0ull;
        }
        // long rows to the table
        auto copy_long = [&]() {
            unsigned long long li = lbase_s + (ex >> 16);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (best[q] <= (uint32_t)SHORT_MAX) continue;
                const int32_t *row = rowv + (q * NT + (int)threadIdx.x) * t;
                if (li < lt.cap && best[q] <= BOUND_LEN_MASK) {
                    int32_t *dst = lt.rows + li * (uint64_t)t;
                    for (int c = 0; c < t; ++c) dst[c] = row[c];
                    lt.bnd[li] = best[q] | ((uint32_t)jb[q] << BOUND_LEN_BITS);
                    lt.blo[li] = lob[q];
                } else {
                    atomicOr(fail, 1u);
                }
                ++li;
            }
        };
        if (!write || ntot == 0) {
            __syncthreads();
            if (ltot) copy_long();
            __syncthreads();
            continue;
        }
        // survivors in rounds of CCAP rows: list, then one coalesced run (the
        // list needs only this batch's total; the output base arrives with
        // the first round's barrier)
        for (uint32_t rb = 0; rb < ntot; rb += CCAP) {
            const uint32_t re = min(ntot, rb + (uint32_t)CCAP);
            // each thread lists its survivors as (local row, candidate
            // position); the values are then fetched with the loads spread
            // over all threads instead of one serial chain per thread
            uint32_t i = ex & 0xffffu;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int lr = q * NT + (int)threadIdx.x;
                if (rb == 0 && mask[q]) lobs[lr] = lob[q];
                for (uint32_t m = mask[q]; m && i < re; m &= m - 1) {
                    if (i >= rb) comp_r[i - rb] = (uint16_t)(lr | ((__ffs(m) - 1) << 10));
                    ++i;
                }
            }
            __syncthreads();
            if (rb == 0 && ltot) copy_long();
            const uint32_t nr0 = re - rb;
            {   // four loads in flight per thread (shared reads first, then the list loads)
                uint32_t r = threadIdx.x;
                for (; r + 3 * NT < nr0; r += 4 * NT) {
                    uint32_t idx[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t e = comp_r[r + j * NT];
                        idx[j] = lobs[e & 1023u] + (e >> 10);
                    }
                    int32_t v[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) v[j] = __ldg(a.ci + idx[j]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) comp_w[r + j * NT] = v[j];
                }
                for (; r < nr0; r += NT) {
                    const uint32_t e = comp_r[r];
                    comp_w[r] = __ldg(a.ci + lobs[e & 1023u] + (e >> 10));
                }
            }
            __syncthreads();
            const uint64_t base = base_s;
            const uint64_t room = cap > base ? cap - base : 0;
            const uint32_t nrow = (uint32_t)min((uint64_t)ntot, room);
            int32_t *dst = out + (base + rb) * (uint64_t)W1;
            const uint32_t nr = nrow > rb ? min(re, nrow) - rb : 0u;
            if (rs < rpw) {
                // four rows per lane per iteration: the shared reads of all
                // four are issued before the first store
                const uint32_t step = (uint32_t)(NW * rpw);
                uint32_t r = (uint32_t)(warp * rpw + rs);
                for (; r + 3 * step < nr; r += 4 * step) {
                    int32_t v[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t rr = r + j * step;
                        v[j] = src_col == t ? comp_w[rr] : rowv[(int)(comp_r[rr] & 1023u) * t + src_col];
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[(uint64_t)(r + j * step) * W1 + oc] = v[j];
                }
                for (; r < nr; r += step) {
                    const int32_t val = src_col == t ? comp_w[r] : rowv[(int)(comp_r[r] & 1023u) * t + src_col];
                    dst[(uint64_t)r * W1 + oc] = val;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace gsi

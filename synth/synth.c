/*
 * Seeded synthetic inputs for the subgraph-isomorphism path: data graphs
 * (Erdos-Renyi, R-MAT), vertex/edge labels (Zipf, uniform) and query graphs
 * (random walks, fixed shapes).  This module holds none of the matching
 * method's arithmetic; it only draws inputs, and both the CUDA library and
 * the CPU oracle consume what it returns.
 *
 * Every random number is a pure function of (seed, stream, counter):
 * splitmix64's output mix applied to a unique 64-bit counter.  Results are
 * therefore identical for any thread count and on any host.
 *
 * The query generator follows the paper's recipe (Sec. VIII-A): walk from a
 * random vertex until |V(Q)| distinct vertices are visited; the visited
 * vertices, the traversed edges and their labels form the query.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

/* ------------------------------------------------------------------ RNG */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* One draw: a unique counter built from seed, stream and index. */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t idx) {
    return mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + idx);
}
static inline double draw_unit(uint64_t seed, uint64_t stream, uint64_t idx) {
    return (double)(draw(seed, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}
static inline uint64_t draw_below(uint64_t seed, uint64_t stream, uint64_t idx, uint64_t bound) {
    /* multiply-shift on the top 32 bits; bound < 2^32 in every use */
    return ((draw(seed, stream, idx) >> 32) * bound) >> 32;
}

enum {
    ST_ER = 1, ST_RMAT = 2, ST_PERM = 3, ST_ELAB = 4, ST_VLAB = 5,
    ST_QSTART = 6, ST_QWALK = 7, ST_QDENSE = 8, ST_QSIZE = 9, ST_SHAPE = 10
};

/* ------------------------------------------------- parallel radix sort */
typedef struct { uint64_t key, val; } kv_t;

typedef struct {
    kv_t *src, *dst;
    int64_t lo, hi;
    int shift, by_val;
    int64_t *hist;            /* [nthreads][256] */
    int tid, nthreads;
    pthread_barrier_t *bar;
} rs_arg_t;

static void *rs_worker(void *p) {
    rs_arg_t *a = (rs_arg_t *)p;
    int64_t *h = a->hist + (int64_t)a->tid * 256;
    memset(h, 0, 256 * sizeof(int64_t));
    for (int64_t i = a->lo; i < a->hi; ++i) {
        uint64_t k = a->by_val ? a->src[i].val : a->src[i].key;
        h[(k >> a->shift) & 255]++;
    }
    pthread_barrier_wait(a->bar);
    if (a->tid == 0) {           /* bin-major, thread-minor exclusive scan: stable */
        int64_t run = 0;
        for (int b = 0; b < 256; ++b)
            for (int t = 0; t < a->nthreads; ++t) {
                int64_t c = a->hist[(int64_t)t * 256 + b];
                a->hist[(int64_t)t * 256 + b] = run;
                run += c;
            }
    }
    pthread_barrier_wait(a->bar);
    for (int64_t i = a->lo; i < a->hi; ++i) {
        uint64_t k = a->by_val ? a->src[i].val : a->src[i].key;
        a->dst[h[(k >> a->shift) & 255]++] = a->src[i];
    }
    return NULL;
}

/* Stable LSD sort of x[0..n) by key (or by val) over the low `bits` bits. */
static void radix_sort_kv(kv_t *x, int64_t n, int bits, int by_val, int nthreads) {
    if (n <= 1) return;
    if (nthreads < 1) nthreads = 1;
    if (n < 65536) nthreads = 1;
    kv_t *tmp = (kv_t *)malloc((size_t)n * sizeof(kv_t));
    int64_t *hist = (int64_t *)malloc((size_t)nthreads * 256 * sizeof(int64_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    rs_arg_t *args = (rs_arg_t *)malloc(sizeof(rs_arg_t) * nthreads);
    pthread_barrier_t bar;
    kv_t *a = x, *b = tmp;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        pthread_barrier_init(&bar, NULL, (unsigned)nthreads);
        for (int t = 0; t < nthreads; ++t) {
            args[t].src = a; args[t].dst = b;
            args[t].lo = n * t / nthreads; args[t].hi = n * (t + 1) / nthreads;
            args[t].shift = 8 * p; args[t].by_val = by_val;
            args[t].hist = hist; args[t].tid = t; args[t].nthreads = nthreads;
            args[t].bar = &bar;
        }
        for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, rs_worker, &args[t]);
        rs_worker(&args[0]);
        for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
        pthread_barrier_destroy(&bar);
        kv_t *s = a; a = b; b = s;
    }
    if (a != x) memcpy(x, a, (size_t)n * sizeof(kv_t));
    free(tmp); free(hist); free(th); free(args);
}

static int bits_for(uint64_t maxv) {
    int b = 0;
    while (b < 64 && (maxv >> b)) ++b;
    return b < 1 ? 1 : b;
}

/* --------------------------------------------- parallel edge sampling */
typedef struct {
    uint64_t seed; int kind;          /* 0 = ER, 1 = R-MAT */
    int32_t n; int scale; double a, b, c;
    uint64_t idx0; int64_t lo, hi;    /* draw indices idx0+lo .. idx0+hi */
    kv_t *out;                        /* out[i - lo] : key or UINT64_MAX for self-loop */
} samp_arg_t;

static void *samp_worker(void *p) {
    samp_arg_t *s = (samp_arg_t *)p;
    for (int64_t i = s->lo; i < s->hi; ++i) {
        uint64_t idx = s->idx0 + (uint64_t)i;
        uint64_t u, v;
        if (s->kind == 0) {
            u = draw_below(s->seed, ST_ER, 2 * idx, (uint64_t)s->n);
            v = draw_below(s->seed, ST_ER, 2 * idx + 1, (uint64_t)s->n);
        } else {
            /* R-MAT: one quadrant choice per level, most significant bit first */
            u = 0; v = 0;
            double ab = s->a + s->b, abc = s->a + s->b + s->c;
            for (int l = 0; l < s->scale; ++l) {
                double r = draw_unit(s->seed, ST_RMAT, idx * 64 + (uint64_t)l);
                u <<= 1; v <<= 1;
                if (r < s->a) { }
                else if (r < ab) { v |= 1; }
                else if (r < abc) { u |= 1; }
                else { u |= 1; v |= 1; }
            }
        }
        kv_t e;
        e.val = idx;
        if (u == v) e.key = UINT64_MAX;
        else e.key = u < v ? (u << 32) | v : (v << 32) | u;
        s->out[i] = e;
    }
    return NULL;
}

static void sample_batch(uint64_t seed, int kind, int32_t n, int scale, double a, double b, double c,
                         uint64_t idx0, int64_t count, kv_t *out, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    samp_arg_t *args = (samp_arg_t *)malloc(sizeof(samp_arg_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        samp_arg_t *s = &args[t];
        s->seed = seed; s->kind = kind; s->n = n; s->scale = scale; s->a = a; s->b = b; s->c = c;
        s->idx0 = idx0; s->lo = count * t / nthreads; s->hi = count * (t + 1) / nthreads; s->out = out;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, samp_worker, &args[t]);
    samp_worker(&args[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(args);
}

/*
 * Draw undirected pairs until `m` distinct non-loop pairs exist; keep the first
 * `m` distinct pairs in draw order; apply a seeded vertex permutation
 * (optional); return them sorted by (min, max) with src < dst.
 * Returns m on success, -1 on allocation failure.
 */
static int64_t sample_graph(uint64_t seed, int kind, int32_t n, int scale, double a, double b, double c,
                            int64_t m, int permute, int nthreads, int32_t *src, int32_t *dst) {
    int64_t cap = m + m / 4 + 1024;
    kv_t *pool = (kv_t *)malloc((size_t)cap * 2 * sizeof(kv_t));
    if (!pool) return -1;
    int64_t have = 0;          /* distinct entries kept in pool[0..have) sorted by key */
    uint64_t next_idx = 0;
    /* valid keys are (u << 32 | v) with u, v < n; self-loops carry UINT64_MAX,
       whose low bits differ from every valid key, and are dropped below */
    int keybits = 32 + bits_for((uint64_t)(n > 1 ? n - 1 : 1));
    while (have < m) {
        int64_t want = (m - have) + (m - have) / 8 + 1024;
        if (have + want > 2 * cap) {
            cap = (have + want) / 2 + 1;
            kv_t *np = (kv_t *)realloc(pool, (size_t)cap * 2 * sizeof(kv_t));
            if (!np) { free(pool); return -1; }
            pool = np;
        }
        sample_batch(seed, kind, n, scale, a, b, c, next_idx, want, pool + have, nthreads);
        next_idx += (uint64_t)want;
        int64_t tot = have + want;
        /* order by (key, draw index): draw index first, then stable by key */
        radix_sort_kv(pool, tot, bits_for(next_idx), 1, nthreads);
        radix_sort_kv(pool, tot, keybits, 0, nthreads);
        int64_t w = 0;
        for (int64_t i = 0; i < tot; ++i) {
            if (pool[i].key == UINT64_MAX) continue;
            if (w > 0 && pool[w - 1].key == pool[i].key) continue;
            pool[w++] = pool[i];
        }
        have = w;
    }
    /* first m distinct in draw order */
    radix_sort_kv(pool, have, bits_for(next_idx), 1, nthreads);
    int32_t *perm = NULL;
    if (permute) {
        perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        for (int32_t i = 0; i < n; ++i) perm[i] = i;
        for (int32_t i = n - 1; i > 0; --i) {
            int32_t j = (int32_t)draw_below(seed, ST_PERM, (uint64_t)i, (uint64_t)i + 1);
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    }
    for (int64_t i = 0; i < m; ++i) {
        uint64_t u = pool[i].key >> 32, v = pool[i].key & 0xffffffffull;
        if (perm) { u = (uint64_t)perm[u]; v = (uint64_t)perm[v]; }
        pool[i].key = u < v ? (u << 32) | v : (v << 32) | u;
        pool[i].val = 0;
    }
    radix_sort_kv(pool, m, keybits, 0, nthreads);
    for (int64_t i = 0; i < m; ++i) {
        src[i] = (int32_t)(pool[i].key >> 32);
        dst[i] = (int32_t)(pool[i].key & 0xffffffffull);
    }
    free(perm);
    free(pool);
    return m;
}

int64_t synth_er(uint64_t seed, int32_t n, int64_t m, int32_t nthreads, int32_t *src, int32_t *dst) {
    if (n < 2 || m < 0 || (double)m > (double)n * (n - 1) / 2.0) return -1;
    return sample_graph(seed, 0, n, 0, 0, 0, 0, m, 0, nthreads, src, dst);
}

int64_t synth_rmat(uint64_t seed, int32_t scale, int64_t m, double a, double b, double c,
                   int32_t nthreads, int32_t *src, int32_t *dst) {
    if (scale < 1 || scale > 30 || m < 0) return -1;
    int32_t n = (int32_t)1 << scale;
    if ((double)m > (double)n * (n - 1) / 2.0 * 0.5) return -1;
    return sample_graph(seed, 1, n, scale, a, b, c, m, 1, nthreads, src, dst);
}

/* ------------------------------------------------------------- labels */
void synth_labels_uniform(uint64_t seed, uint64_t stream, int64_t count, int32_t nlabels, int32_t *out) {
    for (int64_t i = 0; i < count; ++i)
        out[i] = (int32_t)draw_below(seed, ST_ELAB * 1000 + stream, (uint64_t)i, (uint64_t)nlabels);
}

/* P(label = l) proportional to (l+1)^-s for l in [0, nlabels). */
void synth_labels_zipf(uint64_t seed, uint64_t stream, int64_t count, int32_t nlabels, double s, int32_t *out) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)nlabels);
    double run = 0;
    for (int32_t l = 0; l < nlabels; ++l) { run += pow((double)(l + 1), -s); cdf[l] = run; }
    for (int32_t l = 0; l < nlabels; ++l) cdf[l] /= run;
    for (int64_t i = 0; i < count; ++i) {
        double r = draw_unit(seed, ST_VLAB * 1000 + stream, (uint64_t)i);
        int32_t lo = 0, hi = nlabels - 1;
        while (lo < hi) { int32_t mid = (lo + hi) / 2; if (cdf[mid] > r) hi = mid; else lo = mid + 1; }
        out[i] = lo;
    }
    free(cdf);
}

/* ----------------------------------------------- adjacency for queries */
/* Per vertex, neighbours sorted by (edge label, neighbour id); vertices are
   also grouped by vertex label for the work bound below. */
typedef struct {
    int32_t n; int64_t m;
    int64_t *start;     /* n+1 */
    int32_t *nbr;       /* 2m */
    int32_t *lab;       /* 2m */
    const int32_t *vlab;
    int32_t nvl;        /* number of vertex labels (max + 1) */
    int64_t *vl_start;  /* nvl+1 */
    int32_t *vl_list;   /* n, vertices grouped by label */
    int32_t *vl_pos;    /* n, index of each vertex inside its label's list */
    int32_t nel;        /* edge labels (max + 1) */
    uint32_t *seg;      /* n*(nel+1): offset of (v, l) inside v's list, same in both orders */
    int32_t *dnbr;      /* 2m: neighbours sorted by (edge label, vertex label, id) */
    int32_t *dvl;       /* 2m: vertex label of dnbr[j] */
} adj_t;

static int cmp_pair(const void *a, const void *b) {
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void *synth_adj_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *elab,
                      const int32_t *vlab) {
    adj_t *g = (adj_t *)calloc(1, sizeof(adj_t));
    g->n = n; g->m = m; g->vlab = vlab;
    g->start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    for (int64_t e = 0; e < m; ++e) { g->start[src[e] + 1]++; g->start[dst[e] + 1]++; }
    for (int32_t v = 0; v < n; ++v) g->start[v + 1] += g->start[v];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(cur, g->start, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        int64_t p = cur[u]++; g->nbr[p] = v; g->lab[p] = elab[e];
        p = cur[v]++; g->nbr[p] = u; g->lab[p] = elab[e];
    }
    /* sort each list by (label, neighbour) */
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) if (g->start[v + 1] - g->start[v] > maxdeg) maxdeg = g->start[v + 1] - g->start[v];
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxdeg + 1));
    for (int32_t v = 0; v < n; ++v) {
        int64_t a = g->start[v], b = g->start[v + 1];
        for (int64_t i = a; i < b; ++i) tmp[i - a] = ((int64_t)g->lab[i] << 32) | (uint32_t)g->nbr[i];
        qsort(tmp, (size_t)(b - a), sizeof(int64_t), cmp_pair);
        for (int64_t i = a; i < b; ++i) { g->lab[i] = (int32_t)(tmp[i - a] >> 32); g->nbr[i] = (int32_t)(tmp[i - a] & 0xffffffff); }
    }
    free(tmp);
    free(cur);
    int32_t maxl = 0;
    for (int32_t v = 0; v < n; ++v) if (vlab[v] > maxl) maxl = vlab[v];
    g->nvl = maxl + 1;
    g->vl_start = (int64_t *)calloc((size_t)g->nvl + 1, sizeof(int64_t));
    g->vl_list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    for (int32_t v = 0; v < n; ++v) g->vl_start[vlab[v] + 1]++;
    for (int32_t l = 0; l < g->nvl; ++l) g->vl_start[l + 1] += g->vl_start[l];
    int64_t *vc = (int64_t *)malloc(sizeof(int64_t) * (size_t)g->nvl);
    memcpy(vc, g->vl_start, sizeof(int64_t) * (size_t)g->nvl);
    g->vl_pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    for (int32_t v = 0; v < n; ++v) {
        int64_t at = vc[vlab[v]]++;
        g->vl_list[at] = v;
        g->vl_pos[v] = (int32_t)(at - g->vl_start[vlab[v]]);
    }
    free(vc);
    /* second order for the work bound: (edge label, vertex label, id) */
    int32_t nel = 0;
    for (int64_t e = 0; e < m; ++e) if (elab[e] + 1 > nel) nel = elab[e] + 1;
    if (nel < 1) nel = 1;
    g->nel = nel;
    g->seg = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * (size_t)(nel + 1) + 4);
    g->dnbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->dvl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxdeg + 1));
    for (int32_t v = 0; v < n; ++v) {
        int64_t a = g->start[v], b = g->start[v + 1];
        uint32_t *sv = g->seg + (size_t)v * (size_t)(nel + 1);
        int64_t j = a;
        for (int32_t l = 0; l <= nel; ++l) {
            while (j < b && g->lab[j] < l) ++j;
            sv[l] = (uint32_t)(j - a);
        }
        for (int32_t l = 0; l < nel; ++l) {
            int64_t lo = a + sv[l], hi = a + sv[l + 1];
            for (int64_t x = lo; x < hi; ++x) key[x - lo] = ((int64_t)vlab[g->nbr[x]] << 32) | (uint32_t)g->nbr[x];
            qsort(key, (size_t)(hi - lo), sizeof(int64_t), cmp_pair);
            for (int64_t x = lo; x < hi; ++x) {
                g->dnbr[x] = (int32_t)(key[x - lo] & 0xffffffff);
                g->dvl[x] = (int32_t)(key[x - lo] >> 32);
            }
        }
    }
    free(key);
    return g;
}

void synth_adj_free(void *p) {
    adj_t *g = (adj_t *)p;
    if (!g) return;
    free(g->start); free(g->nbr); free(g->lab); free(g->vl_start); free(g->vl_list); free(g->vl_pos);
    free(g->seg); free(g->dnbr); free(g->dvl); free(g);
}

int64_t synth_adj_degree(void *p, int32_t v) {
    adj_t *g = (adj_t *)p;
    return g->start[v + 1] - g->start[v];
}

/* [lo, hi) of the neighbours of u with edge label l */
static void adj_seg(const adj_t *g, int32_t u, int32_t l, int64_t *lo_out, int64_t *hi_out) {
    int64_t lo = g->start[u], hi = g->start[u + 1];
    while (lo < hi) { int64_t mid = (lo + hi) / 2; if (g->lab[mid] < l) lo = mid + 1; else hi = mid; }
    int64_t a = lo;
    hi = g->start[u + 1];
    while (lo < hi) { int64_t mid = (lo + hi) / 2; if (g->lab[mid] <= l) lo = mid + 1; else hi = mid; }
    *lo_out = a; *hi_out = lo;
}

/* label of edge {u,v}, or -1 */
static int32_t adj_label(const adj_t *g, int32_t u, int32_t v) {
    for (int64_t i = g->start[u]; i < g->start[u + 1];) {
        int32_t l = g->lab[i];
        int64_t a, b;
        adj_seg(g, u, l, &a, &b);
        int64_t lo = a, hi = b;
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (g->nbr[mid] < v) lo = mid + 1; else hi = mid; }
        if (lo < b && g->nbr[lo] == v) return l;
        i = b;
    }
    return -1;
}

/*
 * Cheap lower bound of the count below: keep every non-leaf query vertex of
 * the spanning tree on the walk's own data vertex and let each leaf take any
 * neighbour of its parent's data vertex with the right edge and vertex
 * labels.  Used to reject a walk before the full count.
 */
static double occurrence_leaf_bound(const adj_t *g, int32_t k, const int32_t *qvlab, const int32_t *qsrc,
                                    const int32_t *qdst, const int32_t *qelab, int32_t qm, const int32_t *occ) {
    int32_t par[32], parlab[32], order[32], nchild[32];
    for (int i = 0; i < k; ++i) { par[i] = -2; nchild[i] = 0; }
    par[0] = -1; order[0] = 0;
    int32_t head = 0, tail = 1;
    while (head < tail) {
        int32_t u = order[head++];
        for (int32_t e = 0; e < qm; ++e) {
            int32_t w = -1;
            if (qsrc[e] == u) w = qdst[e]; else if (qdst[e] == u) w = qsrc[e];
            if (w >= 0 && par[w] == -2) { par[w] = u; parlab[w] = qelab[e]; order[tail++] = w; nchild[u]++; }
        }
    }
    double prod = 1.0;
    for (int32_t u = 1; u < k; ++u) {
        if (par[u] < 0 || nchild[u] > 0) continue;
        int64_t a, b;
        adj_seg(g, occ[par[u]], parlab[u], &a, &b);
        int64_t c = 0;
        for (int64_t j = a; j < b; ++j) c += g->vlab[g->nbr[j]] == qvlab[u];
        prod *= (double)c;
    }
    return prod;
}

/*
 * Work bound used to admit a random-walk query: the number of label-preserving
 * homomorphisms of a BFS spanning tree of Q (rooted at query vertex 0) into G.
 * It is an upper bound on the number of embeddings of Q, computed bottom-up:
 * c_u(v) = [L(v) = L(u)] * prod_{children w} sum_{v' in N(v, L(uw))} c_w(v').
 * Each c_u is kept only over the data vertices carrying u's label.
 */
static double tree_hom_bound_limited(const adj_t *g, int32_t k, const int32_t *qvlab, const int32_t *qsrc,
                                     const int32_t *qdst, const int32_t *qelab, int32_t qm, double stop_above) {
    int32_t par[32], parlab[32], order[32];
    for (int i = 0; i < k; ++i) par[i] = -2;
    par[0] = -1; order[0] = 0;
    int32_t head = 0, tail = 1;
    while (head < tail) {
        int32_t u = order[head++];
        for (int32_t e = 0; e < qm; ++e) {
            int32_t w = -1;
            if (qsrc[e] == u) w = qdst[e]; else if (qdst[e] == u) w = qsrc[e];
            if (w >= 0 && par[w] == -2) { par[w] = u; parlab[w] = qelab[e]; order[tail++] = w; }
        }
    }
    if (tail != k) return -1.0;                   /* disconnected */
    for (int i = 0; i < k; ++i)
        if (qvlab[i] < 0 || qvlab[i] >= g->nvl) return 0.0;
    double *c[32];
    for (int i = 0; i < k; ++i) c[i] = NULL;
    for (int32_t oi = k - 1; oi >= 0; --oi) {
        int32_t u = order[oi];
        int32_t lu = qvlab[u];
        const int32_t *list = g->vl_list + g->vl_start[lu];
        int64_t cnt = g->vl_start[lu + 1] - g->vl_start[lu];
        c[u] = (double *)malloc(sizeof(double) * (size_t)(cnt + 1));
        for (int64_t i = 0; i < cnt; ++i) c[u][i] = 1.0;
        for (int32_t w = 0; w < k; ++w) {
            if (par[w] != u) continue;
            const int32_t lw = qvlab[w];
            const double *cw = c[w];
            const int32_t l = parlab[w];
            if (l < 0 || l >= g->nel) {
                for (int64_t i = 0; i < cnt; ++i) c[u][i] = 0.0;
            } else {
                for (int64_t i = 0; i < cnt; ++i) {
                    if (c[u][i] == 0.0) continue;
                    const int32_t v = list[i];
                    const uint32_t *sv = g->seg + (size_t)v * (size_t)(g->nel + 1);
                    int64_t lo = g->start[v] + sv[l], hi = g->start[v] + sv[l + 1];
                    while (lo < hi) {                        /* first entry with label >= lw */
                        int64_t mid = (lo + hi) / 2;
                        if (g->dvl[mid] < lw) lo = mid + 1; else hi = mid;
                    }
                    double acc = 0;
                    const int64_t end = g->start[v] + sv[l + 1];
                    for (int64_t j = lo; j < end && g->dvl[j] == lw; ++j) acc += cw[g->vl_pos[g->dnbr[j]]];
                    c[u][i] *= acc;
                }
            }
            free(c[w]);
            c[w] = NULL;
        }
    }
    double total = 0;
    int64_t cnt0 = g->vl_start[qvlab[0] + 1] - g->vl_start[qvlab[0]];
    for (int64_t i = 0; i < cnt0; ++i) {
        total += c[0][i];
        if (stop_above > 0 && total > stop_above) break;
    }
    free(c[0]);
    return total;
}

double synth_tree_hom_bound(void *p, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                            const int32_t *qelab, int32_t qm, int32_t nthreads) {
    (void)nthreads;
    return tree_hom_bound_limited((const adj_t *)p, k, qvlab, qsrc, qdst, qelab, qm, 0.0);
}

/*
 * Random-walk query (Sec. VIII-A).  Query vertex ids follow the order of first
 * visit.  Sparse: the distinct edges the walk traversed.  Dense: then add data
 * edges among the visited vertices, in seeded random order, until |E(Q)| >= 2k
 * or none are left.  Returns the number of query edges, or -1 if no walk
 * reached k distinct vertices.  qverts receives the data vertex of each query
 * vertex (one occurrence, so every query has at least one embedding).
 */
int32_t synth_walk_query(void *p, const int32_t *vlab, uint64_t seed, int64_t qindex, int32_t k, int32_t dense,
                         double max_bound, int32_t nthreads, int32_t max_attempts, int32_t min_label,
                         int32_t *qvlab, int32_t *qsrc, int32_t *qdst, int32_t *qelab, int32_t *qverts,
                         double *bound_out, int32_t *attempts_out) {
    adj_t *g = (adj_t *)p;
    
    if (k < 1 || k > 32) return -1;
    if (attempts_out) *attempts_out = 0;
    int32_t maxe = k * (k - 1) / 2;
    uint8_t *has = (uint8_t *)calloc((size_t)k * k, 1);
    if (max_attempts <= 0 || max_attempts > 100000) max_attempts = 100000;
    for (int attempt = 0; attempt < max_attempts; ++attempt) {
        uint64_t ctr = (uint64_t)qindex * 100000 + (uint64_t)attempt;
        int32_t start = (int32_t)draw_below(seed, ST_QSTART, ctr, (uint64_t)g->n);
        if (attempts_out) *attempts_out = attempt + 1;
        if (g->start[start + 1] == g->start[start] && k > 1) continue;
        /* rare-label walks visit only vertices labelled min_label or above */
        if (g->vlab[start] < min_label) continue;
        memset(has, 0, (size_t)k * k);
        int32_t nv = 1, ne = 0, cur = start, curq = 0;
        qverts[0] = start;
        int64_t maxsteps = (min_label > 0 ? 256 : 64) * (int64_t)k;
        for (int64_t st = 0; st < maxsteps && nv < k; ++st) {
            int64_t deg = g->start[cur + 1] - g->start[cur];
            /* counter space per attempt: 1024 steps (4096 for rare-label walks) */
            const uint64_t wctr = min_label > 0 ? ctr * 8192 + (uint64_t)st : ctr * 1024 + (uint64_t)st;
            int64_t pick = (int64_t)draw_below(seed, ST_QWALK, wctr, (uint64_t)deg);
            int32_t nb = g->nbr[g->start[cur] + pick];
            if (g->vlab[nb] < min_label) continue;    /* a step to a frequent label is not taken */
            int32_t nbq = -1;
            for (int32_t i = 0; i < nv; ++i) if (qverts[i] == nb) { nbq = i; break; }
            if (nbq < 0) { nbq = nv; qverts[nv++] = nb; }
            if (!has[curq * k + nbq]) {
                has[curq * k + nbq] = has[nbq * k + curq] = 1;
                qsrc[ne] = curq < nbq ? curq : nbq;
                qdst[ne] = curq < nbq ? nbq : curq;
                qelab[ne] = g->lab[g->start[cur] + pick];
                ++ne;
            }
            cur = nb; curq = nbq;
        }
        if (nv < k) continue;
        if (dense) {
            /* candidate extra edges in (i,j) order, then a seeded shuffle */
            int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxe + 1));
            int32_t *cj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxe + 1));
            int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxe + 1));
            int32_t nc = 0;
            for (int32_t i = 0; i < k; ++i)
                for (int32_t j = i + 1; j < k; ++j) {
                    if (has[i * k + j]) continue;
                    int32_t l = adj_label(g, qverts[i], qverts[j]);
                    if (l >= 0) { ci[nc] = i; cj[nc] = j; cl[nc] = l; ++nc; }
                }
            for (int32_t i = nc - 1; i > 0; --i) {
                int32_t j = (int32_t)draw_below(seed, ST_QDENSE, ctr * 1024 + (uint64_t)i, (uint64_t)i + 1);
                int32_t t;
                t = ci[i]; ci[i] = ci[j]; ci[j] = t;
                t = cj[i]; cj[i] = cj[j]; cj[j] = t;
                t = cl[i]; cl[i] = cl[j]; cl[j] = t;
            }
            for (int32_t i = 0; i < nc && ne < 2 * k; ++i) {
                qsrc[ne] = ci[i]; qdst[ne] = cj[i]; qelab[ne] = cl[i]; ++ne;
                has[ci[i] * k + cj[i]] = has[cj[i] * k + ci[i]] = 1;
            }
            free(ci); free(cj); free(cl);
        }
        for (int32_t i = 0; i < k; ++i) qvlab[i] = g->vlab[qverts[i]];
        if (max_bound > 0 && occurrence_leaf_bound(g, k, qvlab, qsrc, qdst, qelab, ne, qverts) > max_bound) continue;
        double bound = max_bound > 0 ? tree_hom_bound_limited(g, k, qvlab, qsrc, qdst, qelab, ne, max_bound) : 0.0;
        if (max_bound > 0 && bound > max_bound) continue;
        if (bound_out) *bound_out = bound;
        free(has);
        return ne;
    }
    free(has);
    return -1;
}

/*
 * Fixed 4-vertex shapes found as an occurrence in G, with the data labels of
 * the occurrence.  shape: 0 path P4, 1 star K_{1,3}, 2 triangle + pendant,
 * 3 four-cycle C4, 4 K4 minus one edge.  The occurrence is searched from
 * vertices in seeded random order, neighbours ascending.  Returns the number
 * of query edges, or -1 if G holds no occurrence.
 */
static const int32_t SHAPE_E[5][5][2] = {
    {{0, 1}, {1, 2}, {2, 3}, {-1, -1}, {-1, -1}},
    {{0, 1}, {0, 2}, {0, 3}, {-1, -1}, {-1, -1}},
    {{0, 1}, {1, 2}, {0, 2}, {2, 3}, {-1, -1}},
    {{0, 1}, {1, 2}, {2, 3}, {0, 3}, {-1, -1}},
    {{0, 1}, {1, 2}, {0, 2}, {1, 3}, {2, 3}},
};
static const int32_t SHAPE_NE[5] = {3, 3, 4, 4, 5};

static int shape_extend(const adj_t *g, int shape, int32_t *f, int depth) {
    if (depth == 4) return 1;
    /* query vertex `depth` is adjacent to some earlier vertex in every shape */
    int32_t anchor = -1;
    for (int e = 0; e < SHAPE_NE[shape]; ++e) {
        int32_t a = SHAPE_E[shape][e][0], b = SHAPE_E[shape][e][1];
        if (b == depth && a < depth) { anchor = a; break; }
        if (a == depth && b < depth) { anchor = b; break; }
    }
    int32_t av = f[anchor];
    for (int64_t p = g->start[av]; p < g->start[av + 1]; ++p) {
        int32_t w = g->nbr[p];
        int ok = 1;
        for (int i = 0; i < depth; ++i) if (f[i] == w) { ok = 0; break; }
        for (int e = 0; ok && e < SHAPE_NE[shape]; ++e) {
            int32_t a = SHAPE_E[shape][e][0], b = SHAPE_E[shape][e][1];
            int32_t other = a == depth ? b : (b == depth ? a : -1);
            if (other >= 0 && other < depth && adj_label(g, f[other], w) < 0) ok = 0;
        }
        if (!ok) continue;
        f[depth] = w;
        if (shape_extend(g, shape, f, depth + 1)) return 1;
    }
    return 0;
}

int32_t synth_shape_query(void *p, const int32_t *vlab, uint64_t seed, int32_t shape,
                          int32_t *qvlab, int32_t *qsrc, int32_t *qdst, int32_t *qelab, int32_t *qverts) {
    adj_t *g = (adj_t *)p;
    if (shape < 0 || shape > 4) return -1;
    int32_t n = g->n;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) order[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)draw_below(seed, ST_SHAPE, (uint64_t)shape * (1ull << 32) + (uint64_t)i, (uint64_t)i + 1);
        int32_t t = order[i]; order[i] = order[j]; order[j] = t;
    }
    int32_t f[4];
    int found = 0;
    for (int32_t i = 0; i < n && !found; ++i) {
        f[0] = order[i];
        found = shape_extend(g, shape, f, 1);
    }
    free(order);
    if (!found) return -1;
    for (int e = 0; e < SHAPE_NE[shape]; ++e) {
        qsrc[e] = SHAPE_E[shape][e][0];
        qdst[e] = SHAPE_E[shape][e][1];
        qelab[e] = adj_label(g, f[qsrc[e]], f[qdst[e]]);
    }
    for (int i = 0; i < 4; ++i) { qvlab[i] = g->vlab[f[i]]; qverts[i] = f[i]; }
    return SHAPE_NE[shape];
}

/* Query sizes and Poisson arrivals for the workload recipes. */
int32_t synth_uniform_int(uint64_t seed, uint64_t stream, int64_t idx, int32_t lo, int32_t hi) {
    return lo + (int32_t)draw_below(seed, ST_QSIZE * 1000 + stream, (uint64_t)idx, (uint64_t)(hi - lo + 1));
}

double synth_unit(uint64_t seed, uint64_t stream, int64_t idx) {
    return draw_unit(seed, ST_QSIZE * 1000 + stream, (uint64_t)idx);
}

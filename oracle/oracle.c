/*
 * ORACLE -- test infrastructure only.  A plain, slow, obviously correct CPU
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load this library; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * Functions and the passages they follow (Sun et al., "GSI: GPU-friendly
 * Subgraph Isomorphism", arXiv 1906.03420):
 *
 *   oracle_enumerate   Defs. 1-3 (Sec. II-A): all injective maps f: V(Q) -> V(G)
 *                      with L_V(f(u)) = L_V(u) and, for every query edge u1u2,
 *                      f(u1)f(u2) in E(G) with the same edge label.  Matches are
 *                      reported as mappings (one row per f), non-induced.
 *                      Recursive backtracking in BFS order of Q from vertex 0.
 *   oracle_bruteforce  The same definition by exhaustive enumeration of every
 *                      injective map (tiny inputs only); used to pin the above.
 *   oracle_enumerate_hom, oracle_bruteforce_hom
 *                      Sec. VII-A: homomorphism semantics drops injectivity
 *                      (two query vertices may map to one data vertex); the
 *                      same backtracking and exhaustive check without it.
 *   oracle_enumerate_edge, oracle_bruteforce_edge
 *                      Sec. VII-A, edge isomorphism: all injective maps
 *                      h: E(Q) -> E(G) such that h(e) has e's edge label and
 *                      e's pair of endpoint labels, and any two query edges
 *                      that share a query vertex b map to data edges that
 *                      share a data vertex with b's label.  Computed on G
 *                      itself (no line graph): backtracking over query edges,
 *                      each after the first taken among the data edges
 *                      incident to the image of an earlier adjacent edge;
 *                      and the exhaustive check of all m^|E(Q)| maps.
 *                      Rows hold data edge ids (positions in the caller's
 *                      edge list), column j = query edge j.
 *   oracle_signature   Sec. III-A: N = 512-bit vertex signature.  The first
 *                      K = 32 bits hold the vertex label itself (Sec. VII-B
 *                      says single labels are stored directly); the other 480
 *                      bits are 240 two-bit groups.  Each (edge label,
 *                      neighbour label) pair is hashed to a group, whose state
 *                      is 00 / 01 / 11 for 0 / 1 / >= 2 pairs.
 *   oracle_filter      Sec. III-A: v in C(u) iff the labels are equal and
 *                      S(v) & S(u) == S(u) on the 480 group bits.
 *   oracle_join_step   Alg. 3's result for one join iteration: each row m of M
 *                      is extended by every w with w in C(u), w not in m
 *                      (set subtraction = injectivity) and w in N(m[c_j], l_j)
 *                      for every linking edge (c_j, l_j).
 *
 * Readings where the paper is silent or garbled (the same list is kept in the
 * design notes): non-induced matching; mappings, not subgraphs; undirected
 * edges with one label per vertex pair; edge isomorphism constrains only
 * query edges that share a vertex (the method runs the non-induced matching
 * on line graphs), and keeps edge labels, endpoint labels and the label of
 * each shared vertex; the signature hash is MurmurHash3
 * x86_32 (the draft text names MurmurHash 2.0; the published text names no
 * hash) over the 8 little-endian bytes (L_e, L_v') with seed 0x9747B28C, and
 * group index = hash mod 240.
 *
 * Fingerprint of a row set (order independent): count, sum of h(row) mod 2^64
 * and xor of h(row), where h chains splitmix64's output mix over the row:
 * h = 0x243F6A8885A308D3; for each id: h = mix64(h + (uint32)id).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    int32_t n;
    int64_t m;
    int32_t *vlab;
    int64_t *start;   /* n+1 */
    int32_t *nbr;     /* 2m, ascending per vertex */
    int32_t *lab;     /* 2m */
    int32_t *esrc, *edst, *elab;   /* m: the caller's edge list */
    int32_t *inc;     /* 2m: ids of the edges at each vertex (same ranges as
                         nbr), ascending */
} og_t;

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void *oracle_graph_new(int32_t n, int64_t m, const int32_t *vlab, const int32_t *src, const int32_t *dst,
                       const int32_t *elab) {
    og_t *g = (og_t *)calloc(1, sizeof(og_t));
    g->n = n; g->m = m;
    g->vlab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    memcpy(g->vlab, vlab, sizeof(int32_t) * (size_t)n);
    g->start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    for (int64_t e = 0; e < m; ++e) { g->start[src[e] + 1]++; g->start[dst[e] + 1]++; }
    for (int32_t v = 0; v < n; ++v) g->start[v + 1] += g->start[v];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(cur, g->start, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = cur[src[e]]++; g->nbr[p] = dst[e]; g->lab[p] = elab[e];
        p = cur[dst[e]]++; g->nbr[p] = src[e]; g->lab[p] = elab[e];
    }
    free(cur);
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) if (g->start[v + 1] - g->start[v] > maxdeg) maxdeg = g->start[v + 1] - g->start[v];
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxdeg + 1));
    for (int32_t v = 0; v < n; ++v) {
        int64_t a = g->start[v], b = g->start[v + 1];
        for (int64_t i = a; i < b; ++i) tmp[i - a] = ((int64_t)g->nbr[i] << 32) | (uint32_t)g->lab[i];
        qsort(tmp, (size_t)(b - a), sizeof(int64_t), cmp_i64);
        for (int64_t i = a; i < b; ++i) { g->nbr[i] = (int32_t)(tmp[i - a] >> 32); g->lab[i] = (int32_t)(uint32_t)tmp[i - a]; }
    }
    free(tmp);
    g->esrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    g->edst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    g->elab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    g->inc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    if (m > 0) {
        memcpy(g->esrc, src, sizeof(int32_t) * (size_t)m);
        memcpy(g->edst, dst, sizeof(int32_t) * (size_t)m);
        memcpy(g->elab, elab, sizeof(int32_t) * (size_t)m);
    }
    cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(cur, g->start, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {      /* ascending e: each vertex's ids come out sorted */
        g->inc[cur[src[e]]++] = (int32_t)e;
        g->inc[cur[dst[e]]++] = (int32_t)e;
    }
    free(cur);
    return g;
}

void oracle_graph_free(void *p) {
    og_t *g = (og_t *)p;
    if (!g) return;
    free(g->vlab); free(g->start); free(g->nbr); free(g->lab);
    free(g->esrc); free(g->edst); free(g->elab); free(g->inc); free(g);
}

/* Label of edge {u, v} in G, or -1 if there is none. */
static int32_t edge_label(const og_t *g, int32_t u, int32_t v) {
    int64_t lo = g->start[u], hi = g->start[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->nbr[mid] < v) lo = mid + 1; else hi = mid;
    }
    if (lo < g->start[u + 1] && g->nbr[lo] == v) return g->lab[lo];
    return -1;
}

int32_t oracle_edge_label(void *p, int32_t u, int32_t v) { return edge_label((og_t *)p, u, v); }

/* ------------------------------------------------------------ fingerprint */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t row_hash(const int32_t *row, int32_t k) {
    uint64_t h = 0x243F6A8885A308D3ull;
    for (int32_t j = 0; j < k; ++j) h = mix64(h + (uint64_t)(uint32_t)row[j]);
    return h;
}

/* ------------------------------------------------------------------ query */
typedef struct {
    int32_t k;
    int32_t vlab[32];
    int32_t elab[32][32];     /* -1 = no edge */
} oq_t;

static int make_query(oq_t *q, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                      const int32_t *qelab, int32_t qm) {
    if (k < 1 || k > 32) return -1;
    q->k = k;
    for (int i = 0; i < k; ++i) { q->vlab[i] = qvlab[i]; for (int j = 0; j < k; ++j) q->elab[i][j] = -1; }
    for (int32_t e = 0; e < qm; ++e) {
        int32_t a = qsrc[e], b = qdst[e];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return -1;
        if (q->elab[a][b] >= 0) return -1;
        q->elab[a][b] = q->elab[b][a] = qelab[e];
    }
    return 0;
}

/* ------------------------------------------------------------ enumeration */
typedef struct {
    const og_t *g;
    const oq_t *q;
    int32_t order[32];            /* matching order: BFS of Q from vertex 0 */
    int32_t nback[32];            /* earlier-positioned neighbours of order[p] */
    int32_t back_pos[32][32];
    int32_t back_lab[32][32];
    int injective;                /* 1: isomorphism (Defs. 2-3); 0: homomorphism (Sec. VII-A) */
} plan_t;

typedef struct {
    const plan_t *pl;
    int32_t f[32];
    int64_t count;
    uint64_t fp_sum, fp_xor;
    int32_t *out; int64_t max_rows;
} enum_state_t;

static void emit(enum_state_t *s) {
    const oq_t *q = s->pl->q;
    int32_t row[32];
    for (int p = 0; p < q->k; ++p) row[s->pl->order[p]] = s->f[p];
    uint64_t h = row_hash(row, q->k);
    s->fp_sum += h; s->fp_xor ^= h;
    if (s->out && s->count < s->max_rows) memcpy(s->out + s->count * q->k, row, sizeof(int32_t) * (size_t)q->k);
    s->count++;
}

static int feasible(const enum_state_t *s, int p, int32_t w) {
    const plan_t *pl = s->pl;
    const og_t *g = pl->g;
    if (g->vlab[w] != pl->q->vlab[pl->order[p]]) return 0;
    if (pl->injective)
        for (int i = 0; i < p; ++i) if (s->f[i] == w) return 0;             /* injective */
    for (int b = 0; b < pl->nback[p]; ++b)                                   /* every query edge */
        if (edge_label(g, s->f[pl->back_pos[p][b]], w) != pl->back_lab[p][b]) return 0;
    return 1;
}

static void extend(enum_state_t *s, int p) {
    const plan_t *pl = s->pl;
    const og_t *g = pl->g;
    if (p == pl->q->k) { emit(s); return; }
    if (pl->nback[p] == 0) {          /* first vertex of a component: any data vertex */
        for (int32_t w = 0; w < g->n; ++w)
            if (feasible(s, p, w)) { s->f[p] = w; extend(s, p + 1); }
        return;
    }
    int32_t a = s->f[pl->back_pos[p][0]];
    for (int64_t i = g->start[a]; i < g->start[a + 1]; ++i) {
        int32_t w = g->nbr[i];
        if (feasible(s, p, w)) { s->f[p] = w; extend(s, p + 1); }
    }
}

static void make_plan(plan_t *pl, const og_t *g, const oq_t *q) {
    pl->g = g; pl->q = q;
    pl->injective = 1;
    int32_t seen[32] = {0};
    int32_t tail = 0;
    for (int32_t root = 0; root < q->k; ++root) {
        if (seen[root]) continue;
        int32_t head = tail;
        pl->order[tail++] = root; seen[root] = 1;
        while (head < tail) {
            int32_t u = pl->order[head++];
            for (int32_t w = 0; w < q->k; ++w)
                if (q->elab[u][w] >= 0 && !seen[w]) { seen[w] = 1; pl->order[tail++] = w; }
        }
    }
    for (int p = 0; p < q->k; ++p) {
        pl->nback[p] = 0;
        for (int i = 0; i < p; ++i) {
            int32_t l = q->elab[pl->order[i]][pl->order[p]];
            if (l >= 0) { pl->back_pos[p][pl->nback[p]] = i; pl->back_lab[p][pl->nback[p]] = l; pl->nback[p]++; }
        }
    }
}

typedef struct {
    enum_state_t st;
    int64_t *next;              /* shared candidate cursor */
} worker_t;

static void *enum_worker(void *arg) {
    worker_t *w = (worker_t *)arg;
    const og_t *g = w->st.pl->g;
    for (;;) {
        int64_t v = __atomic_fetch_add(w->next, 1, __ATOMIC_RELAXED);
        if (v >= g->n) break;
        if (feasible(&w->st, 0, (int32_t)v)) { w->st.f[0] = (int32_t)v; extend(&w->st, 1); }
    }
    return NULL;
}

/*
 * All embeddings of Q in G.  Returns the exact count (or -1 on invalid
 * query).  Rows (query-id order, k ints each) are written to out for the
 * first max_rows embeddings when out != NULL; rows are only written when
 * nthreads == 1.  fp[0..2] receives (count, sum h, xor h).
 */
static int64_t enumerate_maps(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                              const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows, int32_t nthreads,
                              uint64_t *fp, int injective) {
    const og_t *g = (const og_t *)gp;
    oq_t q;
    if (make_query(&q, k, qvlab, qsrc, qdst, qelab, qm)) return -1;
    plan_t pl;
    make_plan(&pl, g, &q);
    pl.injective = injective;
    int64_t count = 0; uint64_t s = 0, x = 0;
    if (nthreads <= 1) {
        enum_state_t st;
        memset(&st, 0, sizeof st);
        st.pl = &pl; st.out = out; st.max_rows = out ? max_rows : 0;
        extend(&st, 0);
        count = st.count; s = st.fp_sum; x = st.fp_xor;
    } else {
        if (nthreads > 256) nthreads = 256;
        pthread_t th[256];
        worker_t *ws = (worker_t *)calloc((size_t)nthreads, sizeof(worker_t));
        int64_t next = 0;
        for (int t = 0; t < nthreads; ++t) {
            ws[t].st.pl = &pl; ws[t].next = &next;
            pthread_create(&th[t], NULL, enum_worker, &ws[t]);
        }
        for (int t = 0; t < nthreads; ++t) {
            pthread_join(th[t], NULL);
            count += ws[t].st.count; s += ws[t].st.fp_sum; x ^= ws[t].st.fp_xor;
        }
        free(ws);
    }
    if (fp) { fp[0] = (uint64_t)count; fp[1] = s; fp[2] = x; }
    return count;
}

int64_t oracle_enumerate(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                         const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows, int32_t nthreads,
                         uint64_t *fp) {
    return enumerate_maps(gp, k, qvlab, qsrc, qdst, qelab, qm, out, max_rows, nthreads, fp, 1);
}

/* All homomorphisms of Q in G (Sec. VII-A): as oracle_enumerate without
 * injectivity. */
int64_t oracle_enumerate_hom(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                             const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows, int32_t nthreads,
                             uint64_t *fp) {
    return enumerate_maps(gp, k, qvlab, qsrc, qdst, qelab, qm, out, max_rows, nthreads, fp, 0);
}

/* Matching order used by oracle_enumerate (for tests). */
int32_t oracle_order(int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                     const int32_t *qelab, int32_t qm, int32_t *order_out) {
    oq_t q;
    if (make_query(&q, k, qvlab, qsrc, qdst, qelab, qm)) return -1;
    plan_t pl;
    make_plan(&pl, NULL, &q);
    memcpy(order_out, pl.order, sizeof(int32_t) * (size_t)k);
    return 0;
}

/*
 * Exhaustive check of every injective map f: V(Q) -> V(G) (n!/(n-k)! maps),
 * in lexicographic order of (f(0), ..., f(k-1)).  Tiny inputs only.
 */
static int64_t bruteforce_maps(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                               const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows, int injective) {
    const og_t *g = (const og_t *)gp;
    oq_t q;
    if (make_query(&q, k, qvlab, qsrc, qdst, qelab, qm)) return -1;
    int32_t f[32];
    int64_t count = 0;
    int32_t n = g->n;
    if (injective && k > n) return 0;
    for (int i = 0; i < k; ++i) f[i] = 0;
    for (;;) {
        int ok = 1;
        for (int i = 0; i < k && ok && injective; ++i)
            for (int j = i + 1; j < k; ++j) if (f[i] == f[j]) { ok = 0; break; }
        for (int i = 0; i < k && ok; ++i) if (g->vlab[f[i]] != q.vlab[i]) ok = 0;
        for (int i = 0; i < k && ok; ++i)
            for (int j = i + 1; j < k; ++j)
                if (q.elab[i][j] >= 0 && edge_label(g, f[i], f[j]) != q.elab[i][j]) { ok = 0; break; }
        if (ok) {
            if (out && count < max_rows) memcpy(out + count * k, f, sizeof(int32_t) * (size_t)k);
            ++count;
        }
        int i = k - 1;
        while (i >= 0 && f[i] == n - 1) { f[i] = 0; --i; }
        if (i < 0) break;
        f[i]++;
    }
    return count;
}

int64_t oracle_bruteforce(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                          const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows) {
    return bruteforce_maps(gp, k, qvlab, qsrc, qdst, qelab, qm, out, max_rows, 1);
}

/* Every map f: V(Q) -> V(G) (n^k maps) checked against the homomorphism
 * definition (Sec. VII-A).  Tiny inputs only. */
int64_t oracle_bruteforce_hom(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                              const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows) {
    return bruteforce_maps(gp, k, qvlab, qsrc, qdst, qelab, qm, out, max_rows, 0);
}

/* ------------------------------------------------- edge isomorphism (Sec. VII-A) */
typedef struct {
    int32_t qm;
    int32_t a[32], b[32], lab[32];     /* query edge e = {a[e], b[e]}, label lab[e] */
    int32_t la[32], lb[32];            /* endpoint labels of query edge e */
} oqe_t;

static int make_edge_query(oqe_t *q, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                           const int32_t *qelab, int32_t qm) {
    oq_t chk;
    if (qm < 1 || qm > 32) return -1;
    if (make_query(&chk, k, qvlab, qsrc, qdst, qelab, qm)) return -1;   /* ids, loops, repeated pairs */
    q->qm = qm;
    for (int32_t e = 0; e < qm; ++e) {
        q->a[e] = qsrc[e]; q->b[e] = qdst[e]; q->lab[e] = qelab[e];
        q->la[e] = qvlab[qsrc[e]]; q->lb[e] = qvlab[qdst[e]];
    }
    return 0;
}

/* The query vertex edges e and f share, or -1. */
static int32_t query_common(const oqe_t *q, int32_t e, int32_t f) {
    if (e == f) return -1;
    if (q->a[e] == q->a[f] || q->a[e] == q->b[f]) return q->a[e];
    if (q->b[e] == q->a[f] || q->b[e] == q->b[f]) return q->b[e];
    return -1;
}

/* The data vertex edges d and x share, or -1. */
static int32_t data_common(const og_t *g, int32_t d, int32_t x) {
    if (d == x) return -1;
    if (g->esrc[d] == g->esrc[x] || g->esrc[d] == g->edst[x]) return g->esrc[d];
    if (g->edst[d] == g->esrc[x] || g->edst[d] == g->edst[x]) return g->edst[d];
    return -1;
}

/* Edge label and endpoint labels (as an unordered pair) of data edge d equal
 * those of query edge e. */
static int edge_labels_match(const og_t *g, const oqe_t *q, int32_t e, int32_t d) {
    if (g->elab[d] != q->lab[e]) return 0;
    int32_t x = g->vlab[g->esrc[d]], y = g->vlab[g->edst[d]];
    return (x == q->la[e] && y == q->lb[e]) || (x == q->lb[e] && y == q->la[e]);
}

typedef struct {
    const og_t *g;
    const oqe_t *q;
    int32_t order[32];          /* query edges in matching order (BFS over shared vertices) */
    int32_t anchor[32];         /* an earlier position whose edge shares a vertex, -1 if none */
} eplan_t;

typedef struct {
    const eplan_t *pl;
    int32_t h[32];              /* h[p] = image of query edge order[p] */
    int64_t count;
    uint64_t fp_sum, fp_xor;
    int32_t *out; int64_t max_rows;
} estate_t;

static void make_edge_plan(eplan_t *pl, const og_t *g, const oqe_t *q) {
    pl->g = g; pl->q = q;
    int32_t seen[32] = {0};
    int32_t tail = 0;
    for (int32_t root = 0; root < q->qm; ++root) {
        if (seen[root]) continue;
        int32_t head = tail;
        pl->order[tail++] = root; seen[root] = 1;
        while (head < tail) {
            int32_t e = pl->order[head++];
            for (int32_t f = 0; f < q->qm; ++f)
                if (!seen[f] && query_common(q, e, f) >= 0) { seen[f] = 1; pl->order[tail++] = f; }
        }
    }
    for (int32_t p = 0; p < q->qm; ++p) {
        pl->anchor[p] = -1;
        for (int32_t i = 0; i < p && pl->anchor[p] < 0; ++i)
            if (query_common(q, pl->order[i], pl->order[p]) >= 0) pl->anchor[p] = i;
    }
}

static int edge_feasible(const estate_t *s, int32_t p, int32_t d) {
    const eplan_t *pl = s->pl;
    const og_t *g = pl->g;
    const oqe_t *q = pl->q;
    int32_t e = pl->order[p];
    if (!edge_labels_match(g, q, e, d)) return 0;
    for (int32_t i = 0; i < p; ++i) {
        if (s->h[i] == d) return 0;                                  /* injective */
        int32_t b = query_common(q, pl->order[i], e);
        if (b < 0) continue;                                         /* no constraint */
        int32_t bl = b == q->a[e] ? q->la[e] : q->lb[e];             /* label of the shared query vertex */
        int32_t x = data_common(g, s->h[i], d);
        if (x < 0 || g->vlab[x] != bl) return 0;
    }
    return 1;
}

static void edge_emit(estate_t *s) {
    const eplan_t *pl = s->pl;
    int32_t row[32];
    for (int32_t p = 0; p < pl->q->qm; ++p) row[pl->order[p]] = s->h[p];
    uint64_t h = row_hash(row, pl->q->qm);
    s->fp_sum += h; s->fp_xor ^= h;
    if (s->out && s->count < s->max_rows)
        memcpy(s->out + s->count * pl->q->qm, row, sizeof(int32_t) * (size_t)pl->q->qm);
    s->count++;
}

static void edge_extend(estate_t *s, int32_t p) {
    const eplan_t *pl = s->pl;
    const og_t *g = pl->g;
    if (p == pl->q->qm) { edge_emit(s); return; }
    if (pl->anchor[p] < 0) {                 /* first edge of a component: every data edge */
        for (int64_t d = 0; d < g->m; ++d)
            if (edge_feasible(s, p, (int32_t)d)) { s->h[p] = (int32_t)d; edge_extend(s, p + 1); }
        return;
    }
    /* the image shares a vertex with the anchor's image: an edge at one of its ends */
    int32_t an = s->h[pl->anchor[p]];
    int32_t ends[2] = {g->esrc[an], g->edst[an]};
    for (int j = 0; j < 2; ++j)
        for (int64_t i = g->start[ends[j]]; i < g->start[ends[j] + 1]; ++i) {
            int32_t d = g->inc[i];
            if (j == 1 && (g->esrc[d] == ends[0] || g->edst[d] == ends[0])) continue;   /* listed at ends[0] */
            if (edge_feasible(s, p, d)) { s->h[p] = d; edge_extend(s, p + 1); }
        }
}

typedef struct {
    estate_t st;
    int64_t *next;
} eworker_t;

static void *edge_worker(void *arg) {
    eworker_t *w = (eworker_t *)arg;
    const og_t *g = w->st.pl->g;
    for (;;) {
        int64_t d = __atomic_fetch_add(w->next, 1, __ATOMIC_RELAXED);
        if (d >= g->m) break;
        if (edge_feasible(&w->st, 0, (int32_t)d)) { w->st.h[0] = (int32_t)d; edge_extend(&w->st, 1); }
    }
    return NULL;
}

/*
 * All edge-isomorphic matches of Q in G (Sec. VII-A).  Returns the count, or
 * -1 for an invalid query (no edge, more than 32 edges, bad ids, a loop or a
 * repeated pair).  Rows (qm data edge ids each, column j = query edge j) go to
 * out for the first max_rows matches when out != NULL and nthreads == 1.
 * fp[0..2] receives (count, sum h, xor h).
 */
int64_t oracle_enumerate_edge(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                              const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows, int32_t nthreads,
                              uint64_t *fp) {
    const og_t *g = (const og_t *)gp;
    oqe_t q;
    if (make_edge_query(&q, k, qvlab, qsrc, qdst, qelab, qm)) return -1;
    eplan_t pl;
    make_edge_plan(&pl, g, &q);
    int64_t count = 0; uint64_t s = 0, x = 0;
    if (nthreads <= 1) {
        estate_t st;
        memset(&st, 0, sizeof st);
        st.pl = &pl; st.out = out; st.max_rows = out ? max_rows : 0;
        edge_extend(&st, 0);
        count = st.count; s = st.fp_sum; x = st.fp_xor;
    } else {
        if (nthreads > 256) nthreads = 256;
        pthread_t th[256];
        eworker_t *ws = (eworker_t *)calloc((size_t)nthreads, sizeof(eworker_t));
        int64_t next = 0;
        for (int t = 0; t < nthreads; ++t) {
            ws[t].st.pl = &pl; ws[t].next = &next;
            pthread_create(&th[t], NULL, edge_worker, &ws[t]);
        }
        for (int t = 0; t < nthreads; ++t) {
            pthread_join(th[t], NULL);
            count += ws[t].st.count; s += ws[t].st.fp_sum; x ^= ws[t].st.fp_xor;
        }
        free(ws);
    }
    if (fp) { fp[0] = (uint64_t)count; fp[1] = s; fp[2] = x; }
    return count;
}

/*
 * Every map h: E(Q) -> E(G) (m^qm maps, lexicographic in (h(0), ..., h(qm-1)))
 * checked against the edge-isomorphism definition pair by pair.  Tiny inputs
 * only.
 */
int64_t oracle_bruteforce_edge(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                               const int32_t *qelab, int32_t qm, int32_t *out, int64_t max_rows) {
    const og_t *g = (const og_t *)gp;
    oqe_t q;
    if (make_edge_query(&q, k, qvlab, qsrc, qdst, qelab, qm)) return -1;
    if (g->m < qm) return 0;
    int32_t h[32];
    int64_t count = 0;
    for (int32_t e = 0; e < qm; ++e) h[e] = 0;
    for (;;) {
        int ok = 1;
        for (int32_t e = 0; e < qm && ok; ++e) if (!edge_labels_match(g, &q, e, h[e])) ok = 0;
        for (int32_t e = 0; e < qm && ok; ++e)
            for (int32_t f = e + 1; f < qm; ++f) {
                if (h[e] == h[f]) { ok = 0; break; }
                int32_t b = query_common(&q, e, f);
                if (b < 0) continue;
                int32_t x = data_common(g, h[e], h[f]);
                if (x < 0 || g->vlab[x] != qvlab[b]) { ok = 0; break; }
            }
        if (ok) {
            if (out && count < max_rows) memcpy(out + count * qm, h, sizeof(int32_t) * (size_t)qm);
            ++count;
        }
        int32_t i = qm - 1;
        while (i >= 0 && h[i] == g->m - 1) { h[i] = 0; --i; }
        if (i < 0) break;
        h[i]++;
    }
    return count;
}

/* ------------------------------------------------------------- signature */
static inline uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

/* MurmurHash3, x86 32-bit variant (Austin Appleby's published algorithm). */
uint32_t oracle_murmur3_32(const uint8_t *data, int32_t len, uint32_t seed) {
    const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
    uint32_t h = seed;
    int32_t nblocks = len / 4;
    for (int32_t i = 0; i < nblocks; ++i) {
        uint32_t k = (uint32_t)data[4 * i] | ((uint32_t)data[4 * i + 1] << 8) | ((uint32_t)data[4 * i + 2] << 16) |
                     ((uint32_t)data[4 * i + 3] << 24);
        k *= c1; k = rotl32(k, 15); k *= c2;
        h ^= k; h = rotl32(h, 13); h = h * 5u + 0xe6546b64u;
    }
    const uint8_t *tail = data + 4 * nblocks;
    uint32_t k = 0;
    switch (len & 3) {
        case 3: k ^= (uint32_t)tail[2] << 16; /* fall through */
        case 2: k ^= (uint32_t)tail[1] << 8;  /* fall through */
        case 1: k ^= (uint32_t)tail[0];
                k *= c1; k = rotl32(k, 15); k *= c2; h ^= k;
    }
    h ^= (uint32_t)len;
    h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
    return h;
}

#define SIG_WORDS 16
#define SIG_GROUPS 240
#define SIG_SEED 0x9747B28Cu

static uint32_t pair_group(int32_t elabel, int32_t nlabel) {
    uint8_t b[8];
    uint32_t a = (uint32_t)elabel, c = (uint32_t)nlabel;
    for (int i = 0; i < 4; ++i) { b[i] = (uint8_t)(a >> (8 * i)); b[4 + i] = (uint8_t)(c >> (8 * i)); }
    return oracle_murmur3_32(b, 8, SIG_SEED) % SIG_GROUPS;
}

/* Signature from a list of (edge label, neighbour label) pairs. */
static void signature(int32_t vlabel, const int32_t *el, const int32_t *nl, int64_t cnt, uint32_t *sig) {
    int32_t counts[SIG_GROUPS];
    memset(counts, 0, sizeof counts);
    for (int64_t i = 0; i < cnt; ++i) counts[pair_group(el[i], nl[i])]++;
    memset(sig, 0, sizeof(uint32_t) * SIG_WORDS);
    sig[0] = (uint32_t)vlabel;
    for (int gi = 0; gi < SIG_GROUPS; ++gi) {
        uint32_t word = 1 + (uint32_t)gi / 16, bit = 2 * ((uint32_t)gi % 16);
        if (counts[gi] >= 1) sig[word] |= 1u << bit;          /* state 01 */
        if (counts[gi] >= 2) sig[word] |= 1u << (bit + 1);    /* state 11 */
    }
}

/* Data-vertex signatures, vertex-major: sig[v * 16 + w]. */
void oracle_data_signatures(void *gp, uint32_t *sig) {
    const og_t *g = (const og_t *)gp;
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < g->n; ++v) if (g->start[v + 1] - g->start[v] > maxdeg) maxdeg = g->start[v + 1] - g->start[v];
    int32_t *nl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 1));
    for (int32_t v = 0; v < g->n; ++v) {
        int64_t a = g->start[v], d = g->start[v + 1] - a;
        for (int64_t i = 0; i < d; ++i) nl[i] = g->vlab[g->nbr[a + i]];
        signature(g->vlab[v], g->lab + a, nl, d, sig + (int64_t)v * SIG_WORDS);
    }
    free(nl);
}

/* Query-vertex signatures, vertex-major: sig[u * 16 + w]. */
int32_t oracle_query_signatures(int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                                const int32_t *qelab, int32_t qm, uint32_t *sig) {
    oq_t q;
    if (make_query(&q, k, qvlab, qsrc, qdst, qelab, qm)) return -1;
    int32_t el[32], nl[32];
    for (int32_t u = 0; u < k; ++u) {
        int64_t c = 0;
        for (int32_t w = 0; w < k; ++w)
            if (q.elab[u][w] >= 0) { el[c] = q.elab[u][w]; nl[c] = q.vlab[w]; ++c; }
        signature(q.vlab[u], el, nl, c, sig + (int64_t)u * SIG_WORDS);
    }
    return 0;
}

/* C(u) for every query vertex: member[u * n + v] = 1 iff v in C(u).  Returns 0. */
int32_t oracle_filter(void *gp, int32_t k, const int32_t *qvlab, const int32_t *qsrc, const int32_t *qdst,
                      const int32_t *qelab, int32_t qm, uint8_t *member, int64_t *counts) {
    const og_t *g = (const og_t *)gp;
    uint32_t qs[32 * SIG_WORDS];
    if (oracle_query_signatures(k, qvlab, qsrc, qdst, qelab, qm, qs)) return -1;
    uint32_t *ds = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)g->n * SIG_WORDS);
    oracle_data_signatures(gp, ds);
    for (int32_t u = 0; u < k; ++u) {
        counts[u] = 0;
        const uint32_t *su = qs + u * SIG_WORDS;
        for (int32_t v = 0; v < g->n; ++v) {
            const uint32_t *sv = ds + (int64_t)v * SIG_WORDS;
            int ok = sv[0] == su[0];
            for (int w = 1; w < SIG_WORDS && ok; ++w) if ((sv[w] & su[w]) != su[w]) ok = 0;
            member[(int64_t)u * g->n + v] = (uint8_t)ok;
            counts[u] += ok;
        }
    }
    free(ds);
    return 0;
}

/* --------------------------------------------------------------- join step */
/*
 * One join iteration (Alg. 3's result).  M has nrows rows of t ints.  The new
 * column's candidates are inC[w] != 0; linking edges are (col[j], lab[j]),
 * j < d.  Writes rows (m || w) for every row m (in order) and every admissible
 * w (ascending) to out, up to max_rows rows of t+1 ints; returns the count.
 */
int64_t oracle_join_step(void *gp, const int32_t *M, int64_t nrows, int32_t t, const uint8_t *inC,
                         const int32_t *col, const int32_t *lab, int32_t d, int32_t *out, int64_t max_rows) {
    const og_t *g = (const og_t *)gp;
    if (d < 1) return -1;
    int64_t count = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        const int32_t *m = M + r * t;
        int32_t a = m[col[0]];
        for (int64_t i = g->start[a]; i < g->start[a + 1]; ++i) {   /* every w adjacent to m[col[0]] */
            int32_t w = g->nbr[i];
            if (!inC[w]) continue;
            int ok = 1;
            for (int32_t c = 0; c < t && ok; ++c) if (m[c] == w) ok = 0;
            for (int32_t j = 0; j < d && ok; ++j) if (edge_label(g, m[col[j]], w) != lab[j]) ok = 0;
            if (!ok) continue;
            if (out && count < max_rows) {
                memcpy(out + count * (t + 1), m, sizeof(int32_t) * (size_t)t);
                out[count * (t + 1) + t] = w;
            }
            ++count;
        }
    }
    return count;
}

/* Fingerprint of explicit rows (for tests). */
void oracle_fingerprint(const int32_t *rows, int64_t nrows, int32_t k, uint64_t *fp) {
    uint64_t s = 0, x = 0;
    for (int64_t r = 0; r < nrows; ++r) { uint64_t h = row_hash(rows + r * k, k); s += h; x ^= h; }
    fp[0] = (uint64_t)nrows; fp[1] = s; fp[2] = x;
}

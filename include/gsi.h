/*
 * gsi.h -- C ABI of the GB300 (sm_103a) subgraph-isomorphism library.
 *
 * The library computes what Sun et al., "GSI: GPU-friendly Subgraph
 * Isomorphism" (arXiv 1906.03420) defines: all matches of a labelled query
 * graph Q in a labelled data graph G (Defs. 1-3, Sec. II-A), reported as
 * mappings f: V(Q) -> V(G) that are injective, keep vertex labels and map
 * every query edge to a data edge with the same label.  It follows the
 * paper's two phases: signature filtering (Sec. III-A) and one vertex-oriented
 * join iteration per query vertex (Algs. 2-4, Sec. V).  Sec. VII-A's
 * homomorphism semantics is a query option; its edge isomorphism runs through
 * the line-graph calls (gsi_edge_*).
 *
 * Conventions for every call:
 *   - Ids and labels are int32; counts are uint64.  Graphs are undirected and
 *     simple: one edge (and one label) per unordered vertex pair, no loops.
 *   - Input arrays are read during the call and copied; the caller keeps them.
 *   - Objects (gsi_graph, gsi_edge_graph, gsi_result, gsi_batch, gsi_server)
 *     are owned by the library until the matching *_destroy call.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.  Calls return after their results are
 *     ready unless stated otherwise.
 *   - No call throws.  Failures return a status; gsi_last_error() then holds a
 *     message for the calling thread.
 *   - All device work runs in this library's own CUDA kernels for sm_103a;
 *     there is no CPU fallback.  A missing or unusable GPU yields GSI_ECUDA.
 */
#ifndef GSI_H
#define GSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSI_OK = 0,
    GSI_EINVAL = 1,      /* invalid argument: id out of range, self-loop, duplicate
                            edge, disconnected or empty query, k > 32, ... */
    GSI_ENOMEM = 2,      /* the memory budget cannot hold even a one-row tile */
    GSI_ECAPPED = 3,     /* gsi_result_copy: rows were truncated at the row cap;
                            the count stays exact */
    GSI_ETIMEOUT = 4,    /* a wait ran past its limit */
    GSI_ECANCELLED = 5,  /* a served request was cancelled */
    GSI_ECUDA = 6,       /* a CUDA call or kernel failed */
    GSI_EBUSY = 7        /* a served request is not finished yet */
} gsi_status;

typedef struct gsi_graph gsi_graph;
typedef struct gsi_result gsi_result;
typedef struct gsi_server gsi_server;

/* Largest query handled (query vertices are tracked in 32-bit masks). */
#define GSI_MAX_QUERY_VERTICES 32

/* Signature geometry (Sec. III-A): N = 512 bits per vertex; the first K = 32
   bits hold the vertex label; the other 480 bits are 240 two-bit groups. */
#define GSI_SIG_WORDS 16
#define GSI_SIG_GROUPS 240

/* ------------------------------------------------------------------ graph */
typedef struct {
    int32_t device;      /* CUDA device ordinal */
    void *stream;        /* stream for the build */
} gsi_graph_opts;

typedef struct {
    int32_t n;           /* |V(G)| */
    int32_t n_elabels;   /* L: edge labels are 0..L-1 */
    int32_t n_vlabels;   /* distinct vertex labels */
    int64_t m;           /* |E(G)| (undirected) */
    uint64_t device_bytes;   /* bytes held on the device by the graph */
    double build_ms;         /* device time of the build */
    /* device pointers, valid until gsi_graph_destroy (read-only):
       off  uint32[n*L + 1]: N(v,l) = ci[off[v*L+l] .. off[v*L+l+1])
       ci   int32[2m]: neighbour lists; each N(v,l) sorted by (label rank of
            the neighbour, neighbour id)
       cl   uint16[2m]: label rank of ci[p] (index of its label among the
            sorted distinct vertex labels)
       sig  uint32[16*n]: signature word w of vertex v at sig[w*n + v]
            (column-first, Sec. III-A); word 0 is the vertex label */
    const uint32_t *off;
    const int32_t *ci;
    const uint16_t *cl;
    const uint32_t *sig;
} gsi_graph_info;

/*
 * Load G into device memory and build its label-partitioned CSR (the
 * edge-label-partitioned graphs P(G,l) of Sec. IV in the "basic
 * representation": one row-offset entry per (vertex, label)), the per-label
 * edge frequencies freq(l) (Table "Notations"), the column-first signature
 * table (Sec. III-A) and a copy of it grouped by vertex label (vertex ids of
 * each label in ascending order, groups padded to multiples of 32), which the
 * filter reads.
 *   vlab  int32[n]   vertex labels (any int32)
 *   src, dst, elab  int32[m]   edge i = {src[i], dst[i]} with label elab[i] >= 0
 * Errors: GSI_EINVAL for n < 1, m < 0, an id outside [0,n), a self-loop, a
 * negative edge label, 2m >= 2^32, more than 65535 distinct vertex labels, or
 * the same vertex pair given twice;
 * GSI_ECUDA / GSI_ENOMEM for device failures.  *out is set only on GSI_OK.
 */
gsi_status gsi_graph_create(const int32_t *vlab, int32_t n, const int32_t *src, const int32_t *dst,
                            const int32_t *elab, int64_t m, const gsi_graph_opts *opts, gsi_graph **out);
void gsi_graph_destroy(gsi_graph *g);
gsi_status gsi_graph_get_info(const gsi_graph *g, gsi_graph_info *info);
/*
 * Copy the built layout out (host or device destinations; any may be NULL):
 * off uint32[n*L + 1], ci int32[2m], cl uint16[2m], sig uint32[16*n].
 */
gsi_status gsi_graph_export(const gsi_graph *g, uint32_t *off, int32_t *ci, uint16_t *cl, uint32_t *sig);
/* freq(l) for l in [0, L): number of undirected edges with label l. */
gsi_status gsi_graph_label_freq(const gsi_graph *g, uint64_t *freq, int32_t max_labels);

/* ------------------------------------------------------------------ query */
typedef struct {
    /* device time (CUDA events on the query's stream) and work, accumulated */
    double filter_ms, join_ms, other_ms;
    uint64_t filter_launches, join_launches, other_launches;
    uint64_t filter_bytes;   /* algorithmic bytes of the filter */
    uint64_t join_bytes;     /* algorithmic bytes of the join steps: per row
                                the row, 16 bytes per linking list (its offset
                                pair and label sub-range), the label
                                sub-lists (the shortest once per candidate
                                slot, with the bitmap word), and 4(t+1) per
                                survivor written */
    uint64_t join_items;     /* candidate slots: sum over rows of the length
                                of the row's shortest linking list restricted
                                to the new vertex's label (a bound at most
                                Alg. 4's) */
    uint64_t tiles;          /* row ranges processed (memory-bounded splits);
                                for batches, work units processed */
    uint64_t peak_bytes;     /* peak intermediate-table bytes */
    uint64_t kernels;        /* kernels launched by this library */
    uint64_t host_driven;    /* queries run host-driven (requested or after an
                                arena overflow) */
    uint64_t cand[GSI_MAX_QUERY_VERTICES];   /* |C(u)| per query vertex */
    int32_t order[GSI_MAX_QUERY_VERTICES];   /* join order (query vertex ids) */
    int32_t k;
    uint64_t join_bytes_listwise;   /* join_bytes under the whole-list model:
                                       each linking list N(v,l) read whole,
                                       8 bytes to locate it, one 4-byte bitmap
                                       probe per candidate slot (device-driven
                                       path of gsi_query_run, when asked by
                                       gsi_query_opts.listwise_bytes) */
    double batch_ms;         /* batches: device time of the batch kernel
                                alone (included in join_ms, which also holds
                                queries rerun on the plain path) */
    uint64_t batch_bytes;    /* batches: the batch kernel's share of
                                join_bytes */
} gsi_stats;

/* Query semantics.  GSI_ISOMORPHISM: Defs. 2-3 (injective maps).
 * GSI_HOMOMORPHISM: Sec. VII-A, the set subtraction of Alg. 3 dropped (two
 * query vertices may map to one data vertex); the filter then uses only the
 * "at least one" signature states, the "at least two" state being unsound
 * without injectivity.  Batches and servers run isomorphism only. */
typedef enum { GSI_ISOMORPHISM = 0, GSI_HOMOMORPHISM = 1 } gsi_semantics;

typedef struct {
    void *stream;            /* stream for all device work of the query */
    uint64_t row_cap;        /* max embeddings materialised; 0 = no cap.  The
                                count stays exact beyond the cap. */
    uint64_t mem_budget;     /* bytes for intermediate tables; 0 = 40% of the
                                device's memory */
    int32_t count_only;      /* 1: count embeddings, materialise none */
    int32_t semantics;       /* gsi_semantics (0 = isomorphism) */
    const int32_t *order;    /* optional join order (k query vertex ids, each
                                connected to an earlier one); NULL = Alg. 2 */
    gsi_stats *stats;        /* optional: timing and work counters */
    int32_t host_driven;     /* 1: size every step on the host and split row
                                ranges to fit the budget (the path otherwise
                                taken only when the device-driven arena
                                overflows) */
    int32_t listwise_bytes;  /* 1 (with stats): also count the join's bytes
                                under the whole-list model
                                (gsi_stats.join_bytes_listwise), in a kernel
                                variant that is a few percent slower */
    int32_t no_dedup;        /* 1: join without duplicate removal (Sec. VI-B):
                                every row locates its own sub-lists and
                                probes the bitmap alone (no warp groups, no
                                sub-list memo); same results, for measuring
                                what duplicate removal saves */
    int32_t tight_rows;      /* 1: the final rows always move to a buffer of
                                their own size and the table region they were
                                written in is released at once (for callers
                                that copy the rows out or keep many results);
                                0: the result may keep the region (no copy)
                                while held regions stay within a quarter of
                                device memory */
} gsi_query_opts;

/*
 * Find all embeddings of Q in G (Defs. 2-3): filter (Sec. III-A), order by
 * Alg. 2, then one join iteration per remaining query vertex (Alg. 3 with the
 * Alg. 4 upper bound on each row's output).  The steps run device-driven in
 * an arena (one scratch and two table regions, sizes kept on the device, no
 * host wait between steps) of min(mem_budget, 16 GiB) bytes; if a table does
 * not fit, the query is redone with an arena four times larger, up to
 * mem_budget, and past that host-driven, with row ranges halved until each
 * fits.  (A single arena of the whole default budget costs milliseconds per
 * query to reserve; most queries fit the first one.)
 *   qvlab int32[k]; query edges {qsrc[i], qdst[i]} with label qelab[i], i < qm.
 * Q must be connected (the paper assumes so, Sec. II-A), have 1 <= k <= 32
 * vertices, no self-loop and no repeated vertex pair: otherwise GSI_EINVAL.
 * opts may be NULL (defaults).  *out receives a result object on GSI_OK.
 */
gsi_status gsi_query_run(gsi_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc,
                         const int32_t *qdst, const int32_t *qelab, int32_t qm, const gsi_query_opts *opts,
                         gsi_result **out);

/* Exact number of embeddings (also beyond the row cap): the size of the set
 * of subgraph isomorphisms of Def. 3, i.e. the rows of Alg. 2's final table. */
gsi_status gsi_result_count(const gsi_result *r, uint64_t *count);
/* Number of query vertices k (columns of each row). */
gsi_status gsi_result_columns(const gsi_result *r, int32_t *k);
/*
 * Copy up to max_rows materialised embeddings into dst (host or device
 * memory; the library detects which), row-major int32[rows][k], column j =
 * query vertex j: Alg. 2's final table with its columns in query-vertex
 * order (each row is one match f of Def. 3, f(u_j) in column j).  Row order
 * is unspecified.  *rows receives the number copied.  Returns GSI_ECAPPED
 * when fewer rows were materialised than the count (row cap or count-only),
 * GSI_OK otherwise.  Returns when the copy is complete.
 */
gsi_status gsi_result_copy(const gsi_result *r, int32_t *dst, uint64_t max_rows, uint64_t *rows);
/*
 * gsi_result_copy enqueued on `stream` (cudaStream_t, null = the legacy
 * default stream) instead of completed: *rows and the status are known at
 * once, the bytes land when the stream reaches the copy.  dst should be
 * pinned host memory (or device memory) for the copy to run asynchronously.
 * The result must stay alive until the copy has completed: synchronise the
 * stream, or make the stream that produced the result wait for it, before
 * gsi_result_destroy.  Use: copying one query's rows to the host while the
 * next query runs on another stream.
 */
gsi_status gsi_result_copy_async(const gsi_result *r, int32_t *dst, uint64_t max_rows, uint64_t *rows,
                                 void *stream);
/* Releases the result's device memory stream-ordered on the stream it was
   produced on: destroy results before destroying that stream. */
void gsi_result_destroy(gsi_result *r);

/* ------------------------------------------------------- step-level calls */
/*
 * Signature filter alone (Sec. III-A): for every query vertex u, the bitmap
 * of C(u) = { v : L(v) = L(u) and S(v) & S(u) = S(u) } (n bits, bit v of word
 * v/32) and |C(u)|.  bitmaps: uint32[k][ceil(n/32)], counts: uint64[k], both
 * host or device memory.
 */
gsi_status gsi_filter(gsi_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                      const int32_t *qelab, int32_t qm, uint32_t *bitmaps, uint64_t *counts, void *stream);

/* Query-vertex signatures (Sec. III-A), vertex-major uint32[k][16]. */
gsi_status gsi_query_signatures(const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                                const int32_t *qelab, int32_t qm, uint32_t *sig);

/*
 * One join iteration (Alg. 3) on device buffers.  M: int32[R][t] row-major;
 * the new query vertex u has label ulabel and candidate set cand = C(u) as a
 * bitmap (uint32[ceil(n/32)]); a candidate w must carry ulabel and have its
 * bit set.  Linking edges (col[j], lab[j]) for j < d.  Each row's output is
 * bounded by its shortest linking list restricted to ulabel (the Alg. 4
 * bound, chosen per row).  Writes rows (m || w) to out (int32[out_cap][t+1])
 * and the number of rows found to *count (host).  Rows beyond out_cap are
 * counted, not written.  Scratch memory is allocated stream-ordered on
 * `stream`.  Errors: GSI_EINVAL for t < 1, t >= 32, d < 1, d > t, a column
 * outside [0,t) or a label < 0.
 */
gsi_status gsi_join_step(gsi_graph *g, const int32_t *M, uint64_t R, int32_t t, const uint32_t *cand,
                         int32_t ulabel, const int32_t *col, const int32_t *lab, int32_t d, int32_t *out,
                         uint64_t out_cap, uint64_t *count, void *stream);

/*
 * gsi_join_step without any allocation, for callers that may not allocate
 * device memory: a plugin running inside another runtime that owns all device
 * memory and passes it only input and output buffers, a latency-critical path
 * that must never wait on an allocator, or a process under a strict memory
 * quota.  (The paper has no counterpart; it is a deployment variant of the
 * join step above.)  Arguments, results and errors are those of
 * gsi_join_step; the difference is where scratch lives: one file-scope device
 * array of about 14.7 MB, held on every GPU that loads the library until the
 * process exits.  Limits: R <= 2^20 rows and at most 2^28 candidate slots (sum
 * over rows of the row's output bound + 2); larger calls return GSI_EINVAL with
 * a message.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it.  Every call synchronises `stream` and
 * reads sizes back to pageable host memory, so no call may be made while
 * that stream is being captured into a CUDA graph.  Every call shares the
 * array and it keeps the previous call's contents (the survivor counter is
 * cleared per call); calls that overlap on the GPU race on it and must be
 * serialised by the caller.  Calls no allocator.
 */
gsi_status gsi_join_step_noalloc(gsi_graph *g, const int32_t *M, uint64_t R, int32_t t, const uint32_t *cand,
                                 int32_t ulabel, const int32_t *col, const int32_t *lab, int32_t d, int32_t *out,
                                 uint64_t out_cap, uint64_t *count, void *stream);

/*
 * Alg. 2's matching order (host only, no GPU): cand[u] = |C(u)|, freq[l] for
 * l < n_labels.  order_out[k]: query vertex ids in join order; first_edge[k]:
 * for position p >= 1, the earlier query vertex whose edge to order[p] has the
 * least frequent label (Alg. 4), -1 at p = 0.
 */
gsi_status gsi_plan_order(int32_t k, const int32_t *qsrc, const int32_t *qdst, const int32_t *qelab, int32_t qm,
                          const uint64_t *cand, const uint64_t *freq, int32_t n_labels, int32_t *order_out,
                          int32_t *first_edge);

/* --------------------------------------------------------------- batched */
typedef struct {
    const int32_t *vlab;     /* int32[k] */
    int32_t k;
    const int32_t *src, *dst, *elab;   /* int32[qm] */
    int32_t qm;
} gsi_query_desc;

typedef struct {
    void *stream;
    uint64_t row_cap;        /* per query */
    uint64_t mem_budget;     /* bytes for all intermediate tables of the batch */
    int32_t count_only;
    gsi_stats *stats;        /* optional, accumulated over the batch */
    int32_t seeds_per_item;  /* work-item size: candidates of the first query
                                vertex per (query, range) item; 0 = 32 */
    int32_t item_rows;       /* split size: a work unit whose table has more
                                rows than this after a step keeps this many and
                                queues the rest, in pieces of this many rows,
                                for other CTAs; 0 = 1024, < 0 = never split */
    int32_t isect;           /* how short rows of multi-edge steps intersect
                                their candidates with the other linking lists:
                                GSI_ISECT_BSEARCH (0, default),
                                GSI_ISECT_MERGE, GSI_ISECT_BITMAP */
    int32_t rows_per_thread; /* rows one thread joins per batch of the row
                                pass: 1 or 2 (0 = 2) */
    int32_t block_threads;   /* threads per CTA of the batch kernel: 128 or
                                256 (0 = 256) */
} gsi_batch_opts;

/* Intersection strategies (gsi_batch_opts.isect); all give the same set.
 * BSEARCH searches each candidate in each other linking list; MERGE walks
 * each other list beside the candidates (both sorted); BITMAP searches each
 * element of each other list among the candidates and ANDs the resulting
 * candidate-position masks. */
#define GSI_ISECT_BSEARCH 0
#define GSI_ISECT_MERGE 1
#define GSI_ISECT_BITMAP 2

/*
 * Run nq queries together in one persistent launch (no counterpart in the
 * paper, which runs one query at a time): one filter pass over every query
 * vertex of the batch (Sec. III-A), the Alg. 2 order per query, then work
 * units on shared queues.  A seed unit is a range of one query's first
 * candidate set; a CTA runs every join step (Alg. 3, Alg. 4 bound) on its
 * rows in its own memory slice, and rows past item_rows after a step go back
 * to a queue as new units, so large queries spread over the GPU.  Queries
 * whose tables do not fit a slice (or the batch result area) run again on
 * the plain path of gsi_query_run.  The rows of each result are those
 * gsi_query_run returns, in another order.  outs[i] receives query i's
 * result (or NULL if its status is not GSI_OK); statuses (optional,
 * int32[nq]) receives per-query status.
 */
gsi_status gsi_batch_run(gsi_graph *g, const gsi_query_desc *qs, int32_t nq, const gsi_batch_opts *opts,
                         gsi_result **outs, int32_t *statuses);

/*
 * Autotuner for batched execution (no counterpart in the paper): runs the
 * given calibration batch once per candidate pair (seeds_per_item in
 * {32, 64, 128}) x (item_rows in {512, 1024, 2048}), each twice, and returns
 * the fastest pair in *best_seeds_per_item / *best_item_rows with its time in
 * *best_ms (all optional).  gsi_batch_autotune_full tunes every knob.
 */
gsi_status gsi_batch_autotune(gsi_graph *g, const gsi_query_desc *qs, int32_t nq, const gsi_batch_opts *opts,
                              int32_t *best_seeds_per_item, int32_t *best_item_rows, double *best_ms);
/*
 * The full autotuner: coordinate descent over seeds_per_item {32, 64, 128},
 * item_rows {512, 1024, 2048}, isect {BSEARCH, MERGE, BITMAP} and the block
 * shape (block_threads, rows_per_thread) in {256, 128} x {2, 1}, one knob at
 * a time from the defaults, each candidate timed twice on the calibration
 * batch (wall time of gsi_batch_run).  *best receives opts with the chosen
 * knobs (stream, budget and the rest copied from opts), *best_ms the time of
 * the chosen setting; trials (optional) the number of batch runs made.
 */
gsi_status gsi_batch_autotune_full(gsi_graph *g, const gsi_query_desc *qs, int32_t nq, const gsi_batch_opts *opts,
                                   gsi_batch_opts *best, double *best_ms, int32_t *trials);

/*
 * Prepared batches (no counterpart in the paper): the batch of gsi_batch_run
 * planned once and replayed from a captured CUDA graph.  gsi_batch_prepare
 * validates the queries (statuses, optional, int32[nq]), runs the batched
 * filter once to fix each query's Alg. 2 order and join steps, reserves the
 * batch's device memory (opts->mem_budget, as gsi_batch_run) and captures one
 * pass of device work (the filter and the batch kernel) into a CUDA graph on
 * opts->stream (a private stream when NULL: the legacy stream cannot be
 * captured).  A non-NULL opts->stats only asks the kernels to count
 * algorithmic bytes on every replay (replays take their own stats).
 *
 * gsi_batch_replay launches that graph: every replay recomputes the filter
 * and all join steps on the device and returns results equal to those of
 * gsi_batch_run (rows in another order); what it reuses is host work whose
 * outcome the inputs fix.  outs[i] / statuses[i] as for gsi_batch_run; stats
 * (optional) accumulates the replay's timings and counters.  Replays of one
 * prepared batch must not overlap (they share its device memory); results
 * outlive both later replays and gsi_batch_destroy.
 */
typedef struct gsi_batch gsi_batch;
gsi_status gsi_batch_prepare(gsi_graph *g, const gsi_query_desc *qs, int32_t nq, const gsi_batch_opts *opts,
                             gsi_batch **out, int32_t *statuses);
gsi_status gsi_batch_replay(gsi_batch *b, gsi_result **outs, int32_t *statuses, gsi_stats *stats);
void gsi_batch_destroy(gsi_batch *b);

/* ---------------------------------------------------------------- served */
typedef struct {
    uint64_t mem_budget;     /* device memory for the intermediate tables of
                                the requests running at once (admission
                                budget, see gsi_server_create); 0 = half of
                                the device's free memory at creation */
    int32_t n_streams;       /* slots: worker threads, each with its own stream
                                (0 = 2) */
    uint64_t row_cap;        /* per query */
    int32_t count_only;
    int32_t max_batch;       /* requests a slot takes at once (0 = 2048);
                                1 = one query at a time on the plain path */
    int32_t seeds_per_item;  /* batch work-item size (0 = 32); see
                                gsi_batch_autotune */
    int32_t item_rows;       /* see gsi_batch_opts.item_rows */
    int32_t min_batch;       /* fewer pending requests than this run one at a
                                time on the plain path (every step on all SMs:
                                lower latency than a batch too small to fill
                                the GPU); 0 = 16 */
    int32_t isect;           /* batches: see gsi_batch_opts */
    int32_t rows_per_thread;
    int32_t block_threads;
} gsi_server_opts;

/*
 * A serving loop over a resident graph (continuous batching, no counterpart
 * in the paper).  Each request carries an estimate of its intermediate-table
 * memory (gsi_server_estimate).  A slot takes pending requests in arrival
 * order, up to max_batch, while the batch's reservation -- the sum over its
 * requests of 16 times the estimate or 1 MiB, whichever is larger, and at
 * least 4 GiB in all -- fits what the running batches leave
 * of mem_budget, runs them as one batch on its own stream in a work area of
 * that size (taken from the device's stream-ordered pool), and returns the
 * reservation when the results are out.  Requests arriving while others are
 * on the GPU are admitted as soon as a slot and memory free up, and batches
 * of different slots overlap on the device.  A request too large for the
 * budget on its own runs alone.  With fewer than min_batch requests taken a
 * slot runs them one at a time on the plain path, within the same
 * reservation.  Creation counts the graph's directed edges per (vertex label,
 * vertex label, edge label) on the device for the estimates.  The graph must
 * outlive the server.
 */
gsi_status gsi_server_create(gsi_graph *g, const gsi_server_opts *opts, gsi_server **out);
/*
 * The admission estimate of a query, in bytes: the fewest directed data edges
 * matching one of its query edges by (label of one end, label of the other,
 * edge label), times 8 -- the Alg. 4 preallocation bound of a first join
 * step along that edge before filtering, with two int32 columns per row.
 * Host only (uses the counts made at creation).  GSI_EINVAL for an invalid
 * query.
 */
gsi_status gsi_server_estimate(gsi_server *s, const gsi_query_desc *q, uint64_t *bytes);
/* Enqueue a query (copied).  *ticket identifies it in gsi_server_poll. */
gsi_status gsi_server_submit(gsi_server *s, const gsi_query_desc *q, uint64_t *ticket);
/*
 * Wait up to timeout_ms (0 = do not wait, < 0 = wait until done) for a ticket.
 * GSI_OK: *out receives the result (ownership passes to the caller) and the
 * ticket is retired.  GSI_EBUSY: not finished.  Other codes: the query failed.
 * latency_ms (optional) receives submit-to-completion time.
 */
gsi_status gsi_server_poll(gsi_server *s, uint64_t ticket, int32_t timeout_ms, gsi_result **out,
                           double *latency_ms);
/* Cancel a request that no slot has taken yet: its poll then returns
 * GSI_ECANCELLED.  A request already running finishes normally. */
gsi_status gsi_server_cancel(gsi_server *s, uint64_t ticket);
/* Finish every request already submitted, then stop the slots; results
 * already handed out by gsi_server_poll stay valid, results never polled are
 * destroyed. */
void gsi_server_destroy(gsi_server *s);

/* ------------------------------------------------------ edge isomorphism */
/*
 * Edge isomorphism (Sec. VII-A): maps h: E(Q) -> E(G), injective, such that
 * two query edges that share a query vertex map to data edges that share a
 * data vertex.  The library follows the paper's reduction.
 *   - G becomes its line graph G': vertex i of G' is edge i of G, and two G'
 *     vertices are adjacent when their edges meet at a vertex.
 *   - Q becomes Q' the same way.
 *   - Q' is matched in G' by the ordinary path (gsi_query_run semantics:
 *     non-induced, so query edges that share no vertex are unconstrained).
 *   - A match of Q' is read back as an edge map: row column j holds the data
 *     edge id (position in the caller's edge list) of query edge j.
 * Labels: h(e) must carry e's edge label and e's unordered pair of endpoint
 * labels.  Where two query edges meet at vertex b, their images must meet at
 * a data vertex with b's label.  In G' this becomes:
 *   - a vertex's label is a dense id of the triple (edge label, lower
 *     endpoint-label rank, higher rank), in sorted triple order, where a rank
 *     is the label's index among G's sorted distinct vertex labels;
 *   - an edge's label is the rank of the shared vertex's label.
 * Query labels that G lacks become values nothing in G' carries (-1 for a
 * Q' vertex, INT32_MAX for a Q' edge), so such queries have no matches.
 * The transform runs on the host.  G' has |E(G)| vertices and
 * sum_v deg(v)(deg(v)-1)/2 edges, so it suits graphs without very
 * high-degree vertices.
 */
typedef struct gsi_edge_graph gsi_edge_graph;

/* gsi_edge_graph_create flag: build the transform's tables only, with no
   device graph and no CUDA call (gsi_edge_graph_line and gsi_edge_query_line
   work; gsi_edge_query_run returns GSI_EINVAL). */
#define GSI_EDGE_HOST_ONLY 1

/*
 * Check G, build its line graph on the host and load it on the device with
 * gsi_graph_create (opts as there; flags 0 or GSI_EDGE_HOST_ONLY).  Arrays as
 * for gsi_graph_create; G's arrays are copied and kept for the transform.
 * Errors: GSI_EINVAL for n < 1, m < 1, m >= 2^31, an id outside [0,n), a
 * self-loop, a negative edge label, a repeated vertex pair, more than 65535
 * distinct label triples, or a line graph of 2^31 edges or more;
 * gsi_graph_create's errors for the device build; GSI_ENOMEM when host memory
 * runs out.  *out is set only on GSI_OK.
 */
gsi_status gsi_edge_graph_create(const int32_t *vlab, int32_t n, const int32_t *src, const int32_t *dst,
                                 const int32_t *elab, int64_t m, const gsi_graph_opts *opts, int32_t flags,
                                 gsi_edge_graph **out);
void gsi_edge_graph_destroy(gsi_edge_graph *g);
/*
 * G' copied to host arrays (each may be NULL): lvlab int32[m] (vertex i =
 * edge i of G), and the first min(cap, |E(G')|) edges in lsrc, ldst, lelab.
 * Edges are listed vertex by vertex of G, then by pairs of incident edges in
 * ascending id order (lsrc < ldst).  *ln = |V(G')| = m, *lm = |E(G')|
 * (optional).
 */
gsi_status gsi_edge_graph_line(const gsi_edge_graph *g, int32_t *lvlab, int32_t *lsrc, int32_t *ldst,
                               int32_t *lelab, int64_t cap, int32_t *ln, int64_t *lm);
/*
 * The device line graph G' as an ordinary gsi_graph, owned by g.  Do not
 * destroy it.  It is valid until gsi_edge_graph_destroy; host-only graphs
 * give NULL.  Queries transformed by gsi_edge_query_line can run on it
 * through every call of this header (batches, prepared batches, servers).
 */
gsi_status gsi_edge_graph_device(const gsi_edge_graph *g, gsi_graph **line);
/*
 * Q' of a query against G's label tables (host only).  Q is validated as for
 * gsi_query_run and needs 1 <= qm <= 32 edges.  Outputs (each may be NULL):
 *   - lvlab int32[qm] (vertex j = query edge j);
 *   - the first min(cap, |E(Q')|) edges in lsrc, ldst, lelab, in the order
 *     of gsi_edge_graph_line;
 *   - *lk = qm and *lqm = |E(Q')| (optional).
 * |E(Q')| <= 496.
 */
gsi_status gsi_edge_query_line(const gsi_edge_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc,
                               const int32_t *qdst, const int32_t *qelab, int32_t qm, int32_t *lvlab,
                               int32_t *lsrc, int32_t *ldst, int32_t *lelab, int32_t cap, int32_t *lk,
                               int32_t *lqm);
/*
 * All edge-isomorphic matches of Q in G: Q' matched in G' by gsi_query_run
 * with opts.  opts->semantics must be GSI_ISOMORPHISM.  An opts->order
 * lists query edge ids.  The result has qm columns (column j = data edge id
 * of query edge j); count, row cap and copy behave as for gsi_query_run.
 * Errors: those of gsi_edge_query_line and gsi_query_run; GSI_EINVAL for a
 * host-only graph or another semantics.
 */
gsi_status gsi_edge_query_run(gsi_edge_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc,
                              const int32_t *qdst, const int32_t *qelab, int32_t qm, const gsi_query_opts *opts,
                              gsi_result **out);

/* ------------------------------------------------------------------ misc */
/*
 * Self-test of the library's bounded device waits (no counterpart in the
 * paper): launches the grid barrier used by the one-launch query kernel with
 * one CTA fewer than it waits for, so every wait must give up after
 * spin_limit sleeps (0 = 4096) and the kernel must return.  Returns
 * GSI_ETIMEOUT when the kernel reported the expired wait (the expected
 * outcome), GSI_OK if it did not, GSI_ECUDA on launch failure.
 */
gsi_status gsi_selftest_wait_timeout(int32_t device, uint64_t spin_limit, double *elapsed_ms);

/* Message of the calling thread's last failure ("" if none). */
const char *gsi_last_error(void);
/* Library version string. */
const char *gsi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSI_H */

// Host-side runtime types shared by the C ABI translation units.
#pragma once

#include <cstdint>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace gsi {
// Device memory shared by several results (a batch's result arena); freed
// when the last result referring to it is destroyed.
struct ResultArena {
    int32_t *ptr = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ~ResultArena();
};
}  // namespace gsi

struct gsi_result {
    struct Chunk {
        int32_t *rows;       // device, row-major [nrows][k], column j = query vertex j
        uint64_t nrows;
        bool owned = true;   // false: the rows live in a shared arena
        uint64_t held = 0;   // > 0: a whole table region kept without a tight copy,
                             // counted against the device's held-region allowance
    };
    int32_t k = 0;
    int device = 0;
    uint64_t count = 0;          // exact number of embeddings
    uint64_t materialised = 0;   // rows held in chunks
    std::vector<Chunk> chunks;
    std::shared_ptr<gsi::ResultArena> arena;
    // memory is released stream-ordered on this stream (the one the result was
    // produced on, so the next query on it reuses the memory at once); null
    // selects the library's own release stream
    cudaStream_t stream = nullptr;
    bool own_stream = false;           // true: `stream` is the producing stream
    ~gsi_result();
};

// Body of an extern "C" entry point: no exception crosses the ABI.
#define GSI_API_BEGIN try {
#define GSI_API_END                                                                            \
    }                                                                                          \
    catch (const std::bad_alloc &) {                                                           \
        ::gsi::set_error("host allocation failed");                                            \
        return GSI_ENOMEM;                                                                     \
    }                                                                                          \
    catch (...) {                                                                              \
        ::gsi::set_error("unexpected host exception");                                         \
        return GSI_ECUDA;                                                                      \
    }

namespace gsi {

// Total memory of a device (looked up once per device).
uint64_t device_total_mem(int dev);
// Held table regions: a result may keep the whole region its rows were
// written in (no tight copy) while the regions held on the device stay within
// a quarter of its memory.  hold_region reserves `bytes` of that allowance
// (false when it is used up); release_region returns it.
bool hold_region(int dev, uint64_t bytes);
void release_region(int dev, uint64_t bytes);

struct QueryGraph {
    int32_t k = 0, qm = 0;
    int32_t vlab[GSI_MAX_QUERY_VERTICES];
    int32_t elab[GSI_MAX_QUERY_VERTICES][GSI_MAX_QUERY_VERTICES];   // -1 = no edge
    std::vector<int32_t> src, dst, lab, vl;
};

struct Timer {
    struct Rec {
        cudaEvent_t a, b;
        int kind;            // 0 filter, 1 join kernel, 2 other
    };
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<Rec> recs;
    void begin(int kind);
    void end();
    void resolve(gsi_stats *s);
};

// State of one query's execution (the depth-first join driver).
struct Exec {
    gsi_graph *g = nullptr;
    cudaStream_t st = nullptr;
    int k = 0;
    int32_t order[GSI_MAX_QUERY_VERTICES];
    std::vector<JoinStep> steps;     // steps[t] extends a t-column table
    uint32_t *bitmaps = nullptr;     // [k][nwords], indexed by query vertex id
    unsigned long long *d_scalars = nullptr;   // [0] step count, [1] bytes, [2] items
    uint64_t *h_pinned = nullptr;             // pinned readback words
    unsigned char *h_stage = nullptr;         // pinned upload staging
    size_t h_stage_bytes = 0;
    uint64_t budget = 0, live = 0, peak = 0, tiles = 0;
    uint64_t row_cap = 0;
    int count_only = 0;
    bool listwise = false;           // count whole-list bytes too (gsi_query_opts.listwise_bytes)
    bool nodedup = false;            // join without duplicate removal (gsi_query_opts.no_dedup)
    bool tight_rows = false;         // final rows always to a tight buffer (gsi_query_opts.tight_rows)
    uint64_t join_bytes = 0, join_items = 0, join_bytes_listwise = 0;
    bool stats_read = false;         // the device path read the counters with its status
    uint64_t kernels = 0;            // kernels launched (scan = 3, partition, join, filter, seed = 3)
    bool fell_back = false;          // the query ran host-driven
    gsi_result *res = nullptr;
    gsi_stats *stats = nullptr;
    Timer tm;

    gsi_status run(int t, const int32_t *M, uint64_t R);
    // All steps enqueued with device-resident sizes; *overflow is set when a
    // table or the scratch did not fit its region (nothing is added to res).
    // arena_bytes: scratch + two table regions; *overflow: a table did not
    // fit (or the arena could not be reserved: *no_memory as well)
    gsi_status run_device(uint64_t arena_bytes, bool *overflow, bool *no_memory);
    gsi_status add_chunk(int32_t *rows, uint64_t nrows, uint64_t alloc_rows);
    const uint32_t *cand(const JoinStep &s, int t) const;
};

// One query of a batch, planned on the host after the batched filter.
struct BatchPlan {
    QueryGraph q;
    gsi_status status = GSI_OK;
    bool active = false;             // needs the join (valid, all candidate sets non-empty)
    bool failed = false;             // did not fit the batch arena: rerun on the plain path
    int32_t k = 0;
    int32_t order[GSI_MAX_QUERY_VERTICES];
    std::vector<JoinStep> steps;
    const uint32_t *bitmaps = nullptr;   // [k][nwords] of this query
    uint64_t seed_count = 0;
    uint64_t count = 0;
    std::vector<gsi_result::Chunk> chunks;
    std::shared_ptr<ResultArena> arena;
};

gsi_status plan_for_batch(gsi_graph *g, BatchPlan &p, const uint64_t *cand_counts, const int32_t *ranks);
// Device memory a server slot keeps across batches (allocated once): the
// per-CTA slices and the result staging area.  Results of a batch run with a
// workspace are gathered into one tight buffer that the batch's results
// share, so the workspace is reusable at once.
struct BatchWorkspace {
    unsigned char *arena = nullptr;
    uint64_t arena_bytes = 0;
    int32_t *result = nullptr;
    uint64_t result_bytes = 0;
};

// One k_batch launch (batch.cu): sizing, the device control block and the
// work area.  batch_setup reserves and uploads what stays fixed;
// batch_enqueue_ctl writes the launch's control words (host to device);
// batch_enqueue_kernel resets the query records and runs the kernel (device
// work only when the launch keeps a template, hence capturable);
// batch_collect reads the outcome back into the plans.
struct BatchLaunch {
    int grid = 0, nsm = 152;
    int nt = 256, rpt = 2;                   // block shape of the batch kernel
    size_t sm = 0;
    uint64_t result_bytes = 0, work_bytes = 0, spill_bytes = 0, slices_bytes = 0;
    uint64_t slice = 0, s_bytes = 0, t_bytes = 0, split_rows = 0, sq_cap = 0, rec_cap = 0;
    size_t nq = 0, nitems = 0, ncfg = 0;
    size_t o_q = 0, o_tpl = 0, o_items = 0, o_recs = 0, o_dst = 0, o_sq = 0, o_ready = 0, o_ctl = 0, ctl_bytes = 0;
    unsigned char *ctl = nullptr;            // control block
    unsigned char *arena = nullptr;          // work area: per-CTA slices, then the spill area
    bool own_arena = false;
    unsigned long long *dstats = nullptr;    // algorithmic bytes and candidates (optional)
    bool all_plain = false;                  // the budget holds no slice: every query on the plain path
    bool has_template = false;               // the initial query records also live on the device
    std::vector<unsigned char> q_init;       // initial query records
};
gsi_status batch_setup(BatchLaunch &L, gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &o,
                       uint64_t budget, cudaStream_t st, BatchWorkspace *ws, bool stats, bool keep_template);
gsi_status batch_enqueue_ctl(BatchLaunch &L, int32_t *result, uint64_t result_bytes, cudaStream_t st);
gsi_status batch_enqueue_kernel(BatchLaunch &L, cudaStream_t st);
gsi_status batch_collect(BatchLaunch &L, gsi_graph *g, std::vector<BatchPlan> &plans, int32_t *result,
                         std::shared_ptr<ResultArena> arena, cudaStream_t st, gsi_stats *stats, BatchWorkspace *ws);
void batch_release(BatchLaunch &L, cudaStream_t st);

// The filter outputs and planning inputs of a batch (serve.cu).
struct BatchInputs {
    uint32_t *bitmaps = nullptr;             // [sum of active k][nwords]
    unsigned long long *counts = nullptr;
    FilterPlan fp;
    uint64_t nk = 0;
    std::vector<int32_t> labels;             // query vertex labels (filter bytes)
};
gsi_status batch_plan_all(gsi_graph *g, std::vector<BatchPlan> &plans, gsi_stats *stats, cudaStream_t st,
                          BatchInputs &in);
void batch_inputs_free(BatchInputs &in, cudaStream_t st);
gsi_status batch_finish(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &bo, uint64_t budget,
                        cudaStream_t st, std::vector<gsi_result *> &outs, std::vector<gsi_status> &statuses);
uint64_t batch_budget(const gsi_batch_opts &bo);

gsi_status batch_execute(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &bo,
                         std::vector<gsi_result *> &outs, std::vector<gsi_status> &statuses,
                         BatchWorkspace *ws = nullptr);
gsi_status batch_run_device(gsi_graph *g, std::vector<BatchPlan> &plans, const gsi_batch_opts &o, uint64_t budget,
                            cudaStream_t st, gsi_stats *stats, BatchWorkspace *ws = nullptr);
gsi_status prepare_device(int dev);
gsi_status validate_query(const int32_t *qvlab, int32_t k, const int32_t *qsrc, const int32_t *qdst,
                          const int32_t *qelab, int32_t qm, QueryGraph *q);
void plan_order(const QueryGraph &q, const uint64_t *cand, const uint64_t *freq, int32_t nlabels, int32_t *order,
                int32_t *first);
void make_steps(const QueryGraph &q, const int32_t *order, const int32_t *first, const int32_t *ranks,
                std::vector<JoinStep> &steps);
gsi_status run_query(gsi_graph *g, const QueryGraph &q, const gsi_query_opts &o, gsi_result **out);
// Argument checks of one join-step call (gsi_join_step and its allocation-free
// variant; `who` prefixes the error message).  Fills s with the step (output
// columns in input order, every column tested by the set subtraction), sets
// *count = 0 and *empty when no row can have a survivor (no rows, or a label
// no data vertex or edge carries).
gsi_status join_step_args(const char *who, gsi_graph *g, const int32_t *M, uint64_t R, int32_t t,
                          const uint32_t *cand, int32_t ulabel, const int32_t *col, const int32_t *lab, int32_t d,
                          int32_t *out, uint64_t out_cap, uint64_t *count, JoinStep *s, bool *empty);

}  // namespace gsi

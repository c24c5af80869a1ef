// gsi_join_step_noalloc: the join step for callers that cannot allocate.
//
// Some callers of this library run where allocating device memory is not
// allowed or not affordable: a plugin executing inside another runtime that
// owns every device byte through its own arena and hands the plugin only its
// input and output buffers; a latency-critical serving path that must never
// wait on an allocator (cudaMalloc can synchronise the device, and a
// stream-ordered pool can still have to grow); a process under a strict
// device-memory quota where an allocation in the middle of a request could
// fail.  For them this entry point runs the same kernels as gsi_join_step, but
// every scratch buffer (the row-bound scan, its block sums and per-row bounds,
// the tile partition and the survivor counter) lives in one file-scope __device__ array of fixed
// size.  The caller still provides the input table, the candidate bitmap and
// the output buffer.
//
// Limits: at most 2^20 input rows and 2^28 candidate slots (the sum over rows
// of the row's output bound plus two) per call.  The array takes
// about 14.7 MB on every GPU that loads the library, until the process exits.
// Every call shares it and it keeps the previous call's contents; the
// survivor counter is cleared on each call.  Calls that overlap on the GPU
// (concurrent streams or host threads) race on the array and must be
// serialised by the caller.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "runtime.h"
#include "scan.cuh"

namespace gsi {
namespace {

constexpr uint64_t NA_MAX_ROWS = 1ull << 20;
constexpr uint64_t NA_MAX_SLOTS = 1ull << 28;
// layout in 8-byte words
constexpr uint64_t NA_F = 0;                                              // F: rows + 1
constexpr uint64_t NA_SCAN = NA_F + NA_MAX_ROWS + 1;                      // scan block sums
// block sums (one per scan block, plus the total) and each row's bound as uint32
constexpr uint64_t NA_SCAN_WORDS = (NA_MAX_ROWS + SCAN_NV - 1) / SCAN_NV + 1 + (NA_MAX_ROWS + 1) / 2 + 1;
constexpr uint64_t NA_PART = NA_SCAN + NA_SCAN_WORDS;                     // tile partition
constexpr uint64_t NA_PART_WORDS = NA_MAX_SLOTS / JOIN_NV + 2;
constexpr uint64_t NA_COUNT = NA_PART + NA_PART_WORDS;                    // survivor counter
constexpr uint64_t NA_WORDS = NA_COUNT + 1;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_WORDS];

// Device address of g_noalloc_scratch, looked up once per device (the host
// symbol itself is only a stand-in and must never reach a kernel).
std::mutex g_na_mu;
unsigned long long *g_na_ptr[64];

gsi_status scratch_address(int dev, unsigned long long **out) {
    if (dev < 0 || dev >= 64) {
        set_error("gsi_join_step_noalloc: device ordinal out of range");
        return GSI_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("gsi_join_step_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return GSI_ECUDA;
        }
        g_na_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_na_ptr[dev];
    return GSI_OK;
}

}  // namespace
}  // namespace gsi

using namespace gsi;

extern "C" gsi_status gsi_join_step_noalloc(gsi_graph *g, const int32_t *M, uint64_t R, int32_t t,
                                            const uint32_t *cand, int32_t ulabel, const int32_t *col,
                                            const int32_t *lab, int32_t d, int32_t *out, uint64_t out_cap,
                                            uint64_t *count, void *stream) {
    GSI_API_BEGIN
    JoinStep s;
    bool empty = false;
    GSI_TRY(join_step_args("gsi_join_step_noalloc", g, M, R, t, cand, ulabel, col, lab, d, out, out_cap, count, &s,
                           &empty));
    if (R > NA_MAX_ROWS) {
        set_error("gsi_join_step_noalloc: more than 2^20 input rows (the static scratch limit)");
        return GSI_EINVAL;
    }
    if (join_scan_scratch(R) > (int64_t)NA_SCAN_WORDS) {
        set_error("gsi_join_step_noalloc: scan scratch larger than the static array");
        return GSI_EINVAL;
    }
    if (empty) return GSI_OK;

    GSI_CUDA_TRY(cudaSetDevice(g->device));
    (void)cudaGetLastError();
    unsigned long long *base = nullptr;
    GSI_TRY(scratch_address(g->device, &base));
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *F = reinterpret_cast<uint64_t *>(base + NA_F);
    uint64_t *scr = reinterpret_cast<uint64_t *>(base + NA_SCAN);
    int64_t *part = reinterpret_cast<int64_t *>(base + NA_PART);
    unsigned long long *cnt = base + NA_COUNT;

    GSI_TRY(launch_join_scan(g, M, R, s, F, scr, st));
    uint64_t total = 0;
    GSI_CUDA_TRY(cudaMemcpyAsync(&total, F + R, sizeof total, cudaMemcpyDeviceToHost, st));
    GSI_CUDA_TRY(cudaStreamSynchronize(st));
    if (total > NA_MAX_SLOTS) {
        set_error("gsi_join_step_noalloc: more than 2^28 candidate slots (the static scratch limit)");
        return GSI_EINVAL;
    }
    GSI_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    GSI_TRY(launch_partition(F, R, total, part, st));
    GSI_TRY(launch_join(g, M, R, s, F, total, part, cand, out, out_cap, cnt, out_cap == 0 ? 1 : 0, nullptr, st));
    uint64_t h = 0;
    GSI_CUDA_TRY(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
    GSI_CUDA_TRY(cudaStreamSynchronize(st));
    *count = h;
    return GSI_OK;
    GSI_API_END
}

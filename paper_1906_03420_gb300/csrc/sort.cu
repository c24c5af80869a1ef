// LSD radix sort of 64-bit keys (8-bit digits), used once per graph build to
// order the directed edge entries by (vertex, edge label, neighbour).
//
// Each pass: per-tile digit histograms, one device scan of the bin-major
// histogram, then a stable scatter.  Inside a tile each warp owns a contiguous
// run of keys and walks it 32 keys at a time; __match_any_sync groups lanes
// with equal digits, so ranks follow input order and every pass is stable.
#include "internal.h"
#include "scan.cuh"

namespace gsi {
namespace {

constexpr int RS_NT = 256;
constexpr int RS_WARPS = RS_NT / 32;
constexpr int RS_VT = 16;
constexpr int RS_TILE = RS_NT * RS_VT;
constexpr int RS_WARP_KEYS = 32 * RS_VT;

__global__ void __launch_bounds__(RS_NT) k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                   uint32_t *__restrict__ hist, int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_VT; ++j) {
        int64_t i = base + j * RS_NT + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                                      int64_t n, int shift, const uint32_t *__restrict__ offs,
                                                      int64_t nblocks) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t goff[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_NT) (&wcnt[0][0])[i] = 0;
    goff[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();

    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_WARP_KEYS;
    uint64_t key[RS_VT];
    uint32_t pos[RS_VT];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_VT; ++r) {
        int64_t i = wbase + r * 32 + lane;
        bool valid = i < n;
        key[r] = valid ? in[i] : 0ull;
        uint32_t dig = valid ? (uint32_t)((key[r] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(FULL_MASK, dig);
        uint32_t rank = __popc(peers & lt);
        uint32_t before = valid ? wcnt[warp][dig] : 0u;
        __syncwarp();
        if (valid && rank == 0) wcnt[warp][dig] = before + __popc(peers);
        __syncwarp();
        pos[r] = before + rank;
    }
    __syncthreads();
    {   // exclusive scan over warps for bin threadIdx.x
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_VT; ++r) {
        int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            uint32_t dig = (uint32_t)((key[r] >> shift) & 255u);
            out[(int64_t)goff[dig] + wcnt[warp][dig] + pos[r]] = key[r];
        }
    }
}

}  // namespace

gsi_status radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, cudaStream_t st) {
    if (n <= 1) return GSI_OK;
    if (n >= (int64_t)1 << 32) {
        set_error("radix_sort_u64: more than 2^32 keys");
        return GSI_EINVAL;
    }
    const int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
    const int64_t nh = 256 * nblocks;
    uint32_t *hist = nullptr, *scr = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync(&hist, sizeof(uint32_t) * (size_t)(nh + 1), st));
    GSI_CUDA_TRY(cudaMallocAsync(&scr, sizeof(uint32_t) * (size_t)(scan_blocks(nh) + 1), st));
    uint64_t *a = keys, *b = tmp;
    int passes = (bits + 7) / 8;
    gsi_status rc = GSI_OK;
    for (int p = 0; p < passes && rc == GSI_OK; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<(unsigned)nblocks, RS_NT, 0, st>>>(a, n, shift, hist, nblocks);
        cudaError_t e = device_scan<uint32_t>(LoadProducer<uint32_t>{hist}, nh, StoreWriter<uint32_t>{hist}, scr, st);
        if (e == cudaSuccess) {
            k_rs_scatter<<<(unsigned)nblocks, RS_NT, 0, st>>>(a, b, n, shift, hist, nblocks);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            set_error(std::string("radix sort: ") + cudaGetErrorString(e));
            rc = GSI_ECUDA;
        }
        uint64_t *s = a; a = b; b = s;
    }
    if (rc == GSI_OK && a != keys)
        if (cudaMemcpyAsync(keys, a, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            set_error("radix sort: copy back failed");
            rc = GSI_ECUDA;
        }
    cudaFreeAsync(hist, st);
    cudaFreeAsync(scr, st);
    return rc;
}

}  // namespace gsi

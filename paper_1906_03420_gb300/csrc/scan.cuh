// Device-wide exclusive scan (reduce, spine, down-sweep), no spin waits.
//
// Values come from a producer functor prod(i) and prefixes go to a writer
// functor write(i, prefix) for i in [0, n); write(n, total) is also called.
// Used for the row-offset scan of the graph build, the radix-sort bins, the
// seed compaction and the per-row output bound of each join step (Alg. 4's
// exclusive prefix sum of |N(v'_i, l0)|).
#pragma once

#include "common.cuh"

namespace gsi {

constexpr int SCAN_NT = 256;
constexpr int SCAN_VT = 8;
constexpr int SCAN_NV = SCAN_NT * SCAN_VT;

template <typename T, typename P>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(P prod, int64_t n, T *bsum) {
    __shared__ T wt[SCAN_NT / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_NV;
    T s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_VT; ++j) {
        int64_t i = base + j * SCAN_NT + threadIdx.x;
        if (i < n) s += prod(i);
    }
    T tot = block_sum<SCAN_NT, T>(s, wt);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single block: in-place exclusive scan of bsum[0..nb), bsum[nb] = total.
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_spine(T *bsum, int64_t nb) {
    __shared__ T wt[32];
    T running = 0;
    for (int64_t c = 0; c < nb; c += 1024) {
        int64_t i = c + threadIdx.x;
        T v = i < nb ? bsum[i] : T(0);
        T tot;
        T ex = block_exclusive_scan<1024, T>(v, wt, &tot);
        if (i < nb) bsum[i] = running + ex;
        running += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = running;
}

template <typename T, typename P, typename W>
__global__ void __launch_bounds__(SCAN_NT) k_scan_down(P prod, int64_t n, const T *bsum, int64_t nb, W write) {
    __shared__ T wt[SCAN_NT / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_NV + (int64_t)threadIdx.x * SCAN_VT;
    T vals[SCAN_VT];
    T local = 0;
#pragma unroll
    for (int j = 0; j < SCAN_VT; ++j) {
        int64_t i = base + j;
        vals[j] = i < n ? prod(i) : T(0);
        local += vals[j];
    }
    T tot;
    T ex = block_exclusive_scan<SCAN_NT, T>(local, wt, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_VT; ++j) {
        int64_t i = base + j;
        if (i < n) write(i, ex);
        ex += vals[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) write(n, bsum[nb]);
}

template <typename T, typename W>
__global__ void k_scan_empty(W write) { write(0, T(0)); }

inline int64_t scan_blocks(int64_t n) { return (n + SCAN_NV - 1) / SCAN_NV; }

// Scratch: T[scan_blocks(n) + 1].
template <typename T, typename P, typename W>
cudaError_t device_scan(P prod, int64_t n, W write, T *scratch, cudaStream_t st) {
    if (n <= 0) {
        k_scan_empty<T, W><<<1, 1, 0, st>>>(write);
        return cudaGetLastError();
    }
    int64_t nb = scan_blocks(n);
    k_scan_reduce<T, P><<<(unsigned)nb, SCAN_NT, 0, st>>>(prod, n, scratch);
    k_scan_spine<T><<<1, 1024, 0, st>>>(scratch, nb);
    k_scan_down<T, P, W><<<(unsigned)nb, SCAN_NT, 0, st>>>(prod, n, scratch, nb, write);
    return cudaGetLastError();
}

// Common producers / writers.
template <typename T>
struct LoadProducer {
    const T *a;
    __device__ T operator()(int64_t i) const { return a[i]; }
};
template <typename T>
struct StoreWriter {
    T *out;
    __device__ void operator()(int64_t i, T v) const { out[i] = v; }
};

}  // namespace gsi

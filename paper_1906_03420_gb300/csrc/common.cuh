// Shared device/host helpers of the GSI library (sm_103a).
#pragma once

#include <cstdint>
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "../../include/gsi.h"

namespace gsi {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);

#define GSI_CUDA_TRY(expr)                                                                     \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess) {                                                               \
            ::gsi::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));              \
            return _e == cudaErrorMemoryAllocation ? GSI_ENOMEM : GSI_ECUDA;                   \
        }                                                                                      \
    } while (0)

#define GSI_TRY(expr)                                                                          \
    do {                                                                                       \
        gsi_status _s = (expr);                                                                \
        if (_s != GSI_OK) return _s;                                                           \
    } while (0)

constexpr unsigned FULL_MASK = 0xffffffffu;

__host__ __device__ inline int ceil_log2_bits(uint64_t maxv) {
    int b = 0;
    while (b < 64 && (maxv >> b)) ++b;
    return b < 1 ? 1 : b;
}

// ----------------------------------------------------------- signature
// MurmurHash3 x86_32 (Appleby) of the 8 little-endian bytes (a, b): the key of
// one (edge label, neighbour label) pair, Sec. III-A.
__host__ __device__ inline uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

__host__ __device__ inline uint32_t murmur3_pair(uint32_t a, uint32_t b, uint32_t seed) {
    const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
    uint32_t h = seed;
    uint32_t blk[2] = {a, b};
    for (int i = 0; i < 2; ++i) {
        uint32_t k = blk[i];
        k *= c1;
        k = rotl32(k, 15);
        k *= c2;
        h ^= k;
        h = rotl32(h, 13);
        h = h * 5u + 0xe6546b64u;
    }
    h ^= 8u;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

constexpr uint32_t SIG_SEED = 0x9747B28Cu;

// Group of a pair, and the word / bit of its "at least one" state bit; the
// "at least two" bit is the next one.  Word 0 holds the vertex label.
__host__ __device__ inline uint32_t sig_group(int32_t elabel, int32_t nlabel) {
    return murmur3_pair((uint32_t)elabel, (uint32_t)nlabel, SIG_SEED) % GSI_SIG_GROUPS;
}
__host__ __device__ inline uint32_t sig_word(uint32_t group) { return 1u + group / 16u; }
__host__ __device__ inline uint32_t sig_bit(uint32_t group) { return 2u * (group % 16u); }

// ------------------------------------------------------------ block scan
// Exclusive block-wide scan of one value per thread (NT threads, NT % 32 == 0).
// `warp_tot` must hold NT/32 values.  Returns the exclusive prefix; *total
// receives the block sum.  Contains __syncthreads().
template <int NT, typename T>
__device__ inline T block_exclusive_scan(T v, T *warp_tot, T *total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL_MASK, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) warp_tot[lane] = w;
    }
    __syncthreads();
    T prefix = warp > 0 ? warp_tot[warp - 1] : T(0);
    *total = warp_tot[NW - 1];
    __syncthreads();
    return prefix + x - v;
}

template <int NT, typename T>
__device__ inline T block_sum(T v, T *warp_tot) {
    T tot;
    block_exclusive_scan<NT, T>(v, warp_tot, &tot);
    return tot;
}

__device__ inline unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lower-bound search of x in the ascending list a[0..len): true if present.
__device__ inline bool sorted_contains(const int32_t *__restrict__ a, uint32_t len, int32_t x) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && __ldg(a + lo) == x;
}

}  // namespace gsi

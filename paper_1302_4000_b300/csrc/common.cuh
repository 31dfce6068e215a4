// common.cuh -- shared device helpers of libclusco (status word, reductions, indexing).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/clusco.h"

// Device status word: bit set by kernels, read and cleared by clusco_sync_status().
#define CLUSCO_ST_NONFINITE 1u
#define CLUSCO_ST_TIMEOUT 2u
#define CLUSCO_ST_BOUNDS 4u

__device__ unsigned int g_clusco_status;

__device__ __forceinline__ void set_status(unsigned int bit) { atomicOr(&g_clusco_status, bit); }

// Row-major upper-triangle (a < b) index of the condensed matrix (int64).
__host__ __device__ __forceinline__ int64_t condensed_idx(int64_t a, int64_t b, int64_t N)
{
    return a * N - a * (a + 1) / 2 + (b - a - 1);
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Number of upper-triangle tile pairs (I <= J) for T tiles per side.
__host__ __device__ __forceinline__ int64_t tri_tiles(int64_t T) { return T * (T + 1) / 2; }

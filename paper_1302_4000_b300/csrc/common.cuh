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

// Where the all-pairs kernels put each pair's cRMSD: the dense condensed output
// out[idx - out_base], or, in threshold mode (list != nullptr), an append-only list of the
// pairs with c < tau (NaN never qualifies): list[k] = global condensed index, vals[k] = c for
// k < min(count, cap), in no particular order; *count ends as the number of such pairs even
// when it exceeds cap.
struct PairSink {
    float *out = nullptr;
    int64_t out_base = 0;
    long long *list = nullptr;
    float *vals = nullptr;
    unsigned long long *count = nullptr;
    int64_t cap = 0;
    float tau = 0.f;
};

// Threshold mode, one warp: every lane calls it; lanes with keep append (idx, c) with a single
// atomic for the warp.
__device__ __forceinline__ void sink_append_warp(const PairSink &s, bool keep, int64_t idx, float c)
{
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(s.count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep) {
        const unsigned long long k = base + __popc(m & ((1u << lane) - 1u));
        if (k < (unsigned long long)s.cap) {
            s.list[k] = idx;
            s.vals[k] = c;
        }
    }
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

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

#ifdef CLUSCO_DEBUG_HOOKS
// Test hooks, compiled into the separate debug library only (the production library has none):
// g_debug_skip_arrive makes the forward's TMA producer of CTA 0 skip its first stage (no arrive,
// no copy), so that the bounded waits give up and the status word reports the timeout;
// debug_nd_cap() shrinks the adjoints' near-duplicate queues so that an overflow can be provoked;
// debug_fl_cap() shrinks the exact-digit forward's per-warp lists of flagged pairs, so that the
// refinement's path for the pairs past a list (the flag mask) can be exercised.
__device__ int g_debug_skip_arrive;
inline int64_t &debug_nd_cap()
{
    static int64_t v = 0;
    return v;
}
inline int &debug_fl_cap()
{
    static int v = 0;
    return v;
}
#endif

// Capacity of an adjoint's near-duplicate queue for P pairs (pairs past it are counted, not
// stored, and the overflow is reported through the status word).
inline int64_t nd_cap_for(int64_t P)
{
    int64_t cap = (int64_t)1 << 22;
#ifdef CLUSCO_DEBUG_HOOKS
    if (debug_nd_cap() > 0) cap = debug_nd_cap();
#endif
    return P < cap ? P : cap;
}

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

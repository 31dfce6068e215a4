// pairs_simt.cuh -- the CUDA-core forms over 64x64-model tiles of the upper triangle, condensed
// FP32 output: the plain form (FP32 covariance, FP64 eq. 2 epilogue by the cubic roots) and the
// exact-integer form (24-bit fixed-point covariance summed exactly in int64).
#pragma once
#include "common.cuh"
#include "epilogue.cuh"
#include "prepass.cuh"

namespace clusco {

// Tiles (I, J), I <= J < T, enumerated row by row; C(I) = I*T - I(I-1)/2 tiles precede row I.
__host__ __device__ __forceinline__ int64_t tri_row_start(int64_t I, int64_t T) { return I * T - I * (I - 1) / 2; }

__device__ __forceinline__ void tri_decode(int64_t t, int64_t T, int64_t *I, int64_t *J)
{
    const double b = 2.0 * (double)T + 1.0;
    double disc = b * b - 8.0 * (double)t;
    int64_t i = (int64_t)floor((b - sqrt(fmax(disc, 0.0))) * 0.5);
    if (i < 0) i = 0;
    if (i > T - 1) i = T - 1;
    while (i > 0 && tri_row_start(i, T) > t) --i;
    while (i + 1 < T && tri_row_start(i + 1, T) <= t) ++i;
    *I = i;
    *J = i + (t - tri_row_start(i, T));
}

// One CTA = one 64x64 model tile; 256 threads as 16x16, each 4 A-models x 4 B-models.
// Xk: [Lp][Npad][3] centred FP32 (zero padded). Rows a outside [row_begin, row_end) are skipped;
// each pair's value goes to the sink (dense: out[condensed(a, b) - out_base]; or the list of
// pairs below the threshold).
__global__ void __launch_bounds__(256, 1)
    pairs_simt_kernel(const float *__restrict__ Xk, const double *__restrict__ G64, int64_t N, int64_t Npad, int Lp,
                      int L, int64_t T, int64_t tile0, int64_t row_begin, int64_t row_end, PairSink sink)
{
    __shared__ __align__(16) float As[SIMT_KC][SIMT_TILE * 3];
    __shared__ __align__(16) float Bs[SIMT_KC][SIMT_TILE * 3];
    int64_t I, J;
    tri_decode(tile0 + blockIdx.x, T, &I, &J);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    float acc[4][4][9];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 9; ++e) acc[i][j][e] = 0.f;

    const int64_t a0 = I * SIMT_TILE, b0 = J * SIMT_TILE;
    for (int k0 = 0; k0 < Lp; k0 += SIMT_KC) {
        // cooperative load: 2 x 16 x 192 floats = 1536 float4, 6 per thread
        for (int v = threadIdx.x; v < 2 * SIMT_KC * 48; v += 256) {
            const int which = v / (SIMT_KC * 48);
            const int rem = v % (SIMT_KC * 48);
            const int k = rem / 48, q = rem % 48;
            const int64_t base = which ? b0 : a0;
            const float4 val = *reinterpret_cast<const float4 *>(Xk + ((int64_t)(k0 + k) * Npad + base) * 3 + 4 * q);
            float *dst = which ? &Bs[k][4 * q] : &As[k][4 * q];
            *reinterpret_cast<float4 *>(dst) = val;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < SIMT_KC; ++k) {
            float av[12], bv[12];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 x = *reinterpret_cast<const float4 *>(&As[k][ty * 12 + 4 * q]);
                const float4 y = *reinterpret_cast<const float4 *>(&Bs[k][tx * 12 + 4 * q]);
                av[4 * q] = x.x; av[4 * q + 1] = x.y; av[4 * q + 2] = x.z; av[4 * q + 3] = x.w;
                bv[4 * q] = y.x; bv[4 * q + 1] = y.y; bv[4 * q + 2] = y.z; bv[4 * q + 3] = y.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int al = 0; al < 3; ++al)
#pragma unroll
                        for (int be = 0; be < 3; ++be)
                            acc[i][j][3 * al + be] = fmaf(av[3 * i + al], bv[3 * j + be], acc[i][j][3 * al + be]);
        }
        __syncthreads();
    }

    const double invL = 1.0 / (double)L;
    // every thread runs all 16 (i, j) steps, so that threshold mode's warp appends line up
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = a0 + ty * 4 + i;
        const bool arow = a >= row_begin && a < row_end && a < N;
        const double Ga = arow ? G64[a] : 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t b = b0 + tx * 4 + j;
            const bool ok = arow && b > a && b < N;
            float c = 0.f;
            if (ok) {
                double H[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) H[e] = (double)acc[i][j][e];
                const double Gb = G64[b];
                if (isnan(Ga) || isnan(Gb))
                    c = __int_as_float(0x7fc00000);
                else
                    c = crmsd_plain_fp64(H, Ga, Gb, invL);
            }
            if (!sink.list) {
                if (ok) sink.out[condensed_idx(a, b, N) - sink.out_base] = c;
            } else {
                sink_append_warp(sink, ok && c < sink.tau, ok ? condensed_idx(a, b, N) : 0, c);
            }
        }
    }
}

// The exact-integer form: the same 64 x 64 upper-triangle tiles, each CTA one half (32 B
// models), 256 threads as 16 x 16, each 4 A-models x 2 B-models. The covariance of the 24-bit
// fixed-point coordinates (prepass_int_kernel) is accumulated exactly: every product
// n_a n_b is one 32 x 32 -> 64-bit integer multiply-add (|n| < 2^23, so a sum of L < 2^17
// products cannot overflow int64). Epilogue: the FP32 fast path (crmsd_fast_fp32) on the
// exact covariance rounded to FP32, and, for every pair whose FP32 error bound exceeds
// CLUSCO_TOL_INT, the FP64 Newton refinement (crmsd_refine_newton_fp64) of the exact
// covariance; such pairs are queued per step in shared memory so that whole warps run the
// FP64 arithmetic together.
#ifndef CLUSCO_TOL_INT
#define CLUSCO_TOL_INT 2e-5f  // A: largest FP32 fast-path error accepted for the exact-integer form
#endif
constexpr int INT_MAX_L = 1 << 17;

struct IntFix {
    double H[9];
    int64_t a, b;
    float s;
};

__global__ void __launch_bounds__(256, 1)
    pairs_int_kernel(const int *__restrict__ Xn, const float *__restrict__ scales, const double *__restrict__ G64,
                     int64_t N, int64_t Npad, int Lp, int L, int64_t T, int64_t tile0, int64_t row_begin,
                     int64_t row_end, PairSink sink)
{
    constexpr int HB = SIMT_TILE / 2;  // B models per CTA
    __shared__ __align__(16) int As[SIMT_KC][SIMT_TILE * 3];
    __shared__ __align__(16) int Bs[SIMT_KC][HB * 3];
    __shared__ IntFix q[256];
    __shared__ int qn;
    int64_t I, J;
    tri_decode(tile0 + (blockIdx.x >> 1), T, &I, &J);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (threadIdx.x == 0) qn = 0;

    long long acc[4][2][9];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < 9; ++e) acc[i][j][e] = 0;

    const int64_t a0 = I * SIMT_TILE, b0 = J * SIMT_TILE + HB * (blockIdx.x & 1);
    for (int k0 = 0; k0 < Lp; k0 += SIMT_KC) {
        // cooperative load: 16 x 48 int4 of A and 16 x 24 int4 of B
        for (int v = threadIdx.x; v < SIMT_KC * 72; v += 256) {
            const bool isb = v >= SIMT_KC * 48;
            const int r = isb ? v - SIMT_KC * 48 : v;
            const int w = isb ? 24 : 48;
            const int k = r / w, qd = r % w;
            const int64_t base = isb ? b0 : a0;
            const int4 val = *reinterpret_cast<const int4 *>(Xn + ((int64_t)(k0 + k) * Npad + base) * 3 + 4 * qd);
            int *dst = isb ? &Bs[k][4 * qd] : &As[k][4 * qd];
            *reinterpret_cast<int4 *>(dst) = val;
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < SIMT_KC; ++k) {
            int av[12], bv[6];
#pragma unroll
            for (int qd = 0; qd < 3; ++qd) {
                const int4 x = *reinterpret_cast<const int4 *>(&As[k][ty * 12 + 4 * qd]);
                const int2 y = *reinterpret_cast<const int2 *>(&Bs[k][tx * 6 + 2 * qd]);
                av[4 * qd] = x.x; av[4 * qd + 1] = x.y; av[4 * qd + 2] = x.z; av[4 * qd + 3] = x.w;
                bv[2 * qd] = y.x; bv[2 * qd + 1] = y.y;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int al = 0; al < 3; ++al)
#pragma unroll
                        for (int be = 0; be < 3; ++be)
                            acc[i][j][3 * al + be] += (long long)av[3 * i + al] * (long long)bv[3 * j + be];
        }
        __syncthreads();
    }

    const double invL = 1.0 / (double)L;
    const float invLf = 1.0f / (float)L;
    // every thread runs all 8 (i, j) steps: the queue's barriers and the threshold mode's warp
    // appends line up
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = a0 + ty * 4 + i;
        const bool arow = a >= row_begin && a < row_end && a < N;
        const double Ga = arow ? G64[a] : 0.0;
        float sa[3] = {1.f, 1.f, 1.f};
        if (arow) {
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) sa[ax] = scales[a * 3 + ax];
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int64_t b = b0 + tx * 2 + j;
            const bool ok = arow && b > a && b < N;
            float c = 0.f, sv = 0.f;
            bool flag = false;
            double Hd[9];
            if (ok) {
                const double Gb = G64[b];
                if (isnan(Ga) || isnan(Gb)) {
                    c = __int_as_float(0x7fc00000);
                } else {
                    float Hf[9];
#pragma unroll
                    for (int al = 0; al < 3; ++al)
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            const double sab = (double)sa[al] * (double)scales[b * 3 + be];  // exact
                            Hd[3 * al + be] = sab * (double)acc[i][j][3 * al + be];
                            Hf[3 * al + be] = (float)Hd[3 * al + be];
                        }
                    float ev;
                    c = crmsd_fast_fp32(Hf, (float)Ga, (float)Gb, invLf, &sv, &ev);
                    flag = !(ev <= 2.f * CLUSCO_TOL_INT * c);
                }
            }
            if (flag) {
                const int slot = atomicAdd(&qn, 1);
                IntFix &f = q[slot];
#pragma unroll
                for (int e = 0; e < 9; ++e) f.H[e] = Hd[e];
                f.a = a;
                f.b = b;
                f.s = sv;
            }
            if (!sink.list) {
                if (ok && !flag) sink.out[condensed_idx(a, b, N) - sink.out_base] = c;
            } else {
                sink_append_warp(sink, ok && !flag && c < sink.tau, ok ? condensed_idx(a, b, N) : 0, c);
            }
            __syncthreads();
            const int n = qn;
            __syncthreads();
            if (threadIdx.x == 0) qn = 0;
            if (n) {  // block-uniform: the queued pairs, one per thread, FP64
                const int t = threadIdx.x;
                float cq = 0.f;
                int64_t idx = 0;
                if (t < n) {
                    const IntFix &f = q[t];
                    cq = crmsd_refine_newton_fp64(f.H, G64[f.a], G64[f.b], invL, f.s);
                    idx = condensed_idx(f.a, f.b, N);
                    if (!sink.list) sink.out[idx - sink.out_base] = cq;
                }
                if (sink.list) sink_append_warp(sink, t < n && cq < sink.tau, idx, cq);
            }
            __syncthreads();
        }
    }
}

}  // namespace clusco

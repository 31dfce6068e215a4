// prepass.cuh -- centring, radius-of-gyration sums and operand layout (one warp per model).
//
// Eq. 2 needs centred coordinates, G_A = L R_A^2 = sum_i |a_i - mean(a)|^2 and
// the covariance over centred coordinates. The pre-pass centres every model
// once and writes the operand layout its contraction reads:
//
//  * FP32-SIMT form: Xk[k][a][axis] (atom-major, Npad models x 3 per atom row),
//    k in [0, Lp), zero padded in k and in a; G64[a] = sum of squares (FP64).
//  * tcgen05 forms: K-contiguous planes of 3*N rows x Lp columns, rows grouped
//    32 at a time as 10 models x 3 axes + 2 zero rows, so that a 32-lane TMEM
//    sub-partition always holds whole models:
//        row(a, axis) = 32*(a/10) + 3*(a%10) + axis.
//    BF16_EXACT2: plane 0 = high digit h, plane 1 = low digit l of the 16-bit
//      fixed point value n = round(x/s_axis), n = 256 h + l, |h|,|l| <= 128,
//      s_axis = max|x_axis| / 32639 per model and axis (|n| <= 32639, so that the byte
//      digits below are signed bytes too); G from the same n (exact in int64), so G and
//      the covariance describe the same points.
//    BF16X3: plane 0 = bf16(x), plane 1 = bf16(x - bf16(x)); G from hi + lo.
//    TF32: one FP32 plane holding tf32-rounded x; G from those values.
//    Optionally (xf != nullptr) the centred FP32 coordinates in the same row layout.
//  * exact-integer SIMT form: Xn[k][a][axis] (the FP32-SIMT layout) holding the 24-bit fixed
//    point value n = round(x / s_axis), s_axis = max|x_axis| / (2^23 - 1) per model and axis;
//    G from the same n (exact in int64).
//  The centroid is summed in FP32 per lane and combined in FP64 across lanes;
//  its own rounding error only shifts the model by ~1e-6 A, which changes
//  cRMSD at second order.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace clusco {

constexpr int SIMT_TILE = 64;  // models per SIMT tile side
constexpr int SIMT_KC = 16;    // atoms per SIMT K chunk
constexpr int TC_MA = 40;      // models per tcgen05 A tile (128 rows)
constexpr float Q24 = 8388607.f;  // 2^23 - 1: the 24-bit fixed-point range
constexpr int TC_MB = 20;      // models per tcgen05 B tile (64 rows)

__host__ __device__ __forceinline__ int64_t tc_row(int64_t a, int axis)
{
    return 32 * (a / 10) + 3 * (a % 10) + axis;
}

// Centroid of model a (FP32 lane sums combined in FP64) and a finiteness flag.
__device__ __forceinline__ void model_centroid(const float *__restrict__ x, int L, int lane, float mu[3], bool *finite)
{
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    bool ok = true;
    for (int i = lane; i < L; i += 32) {
        const float v0 = x[3 * i + 0], v1 = x[3 * i + 1], v2 = x[3 * i + 2];
        ok = ok && isfinite(v0) && isfinite(v1) && isfinite(v2);
        s0 += v0;
        s1 += v1;
        s2 += v2;
    }
    const double invL = 1.0 / (double)L;
    mu[0] = (float)(warp_sum_d((double)s0) * invL);
    mu[1] = (float)(warp_sum_d((double)s1) * invL);
    mu[2] = (float)(warp_sum_d((double)s2) * invL);
    *finite = __all_sync(0xffffffffu, ok);
}

// model_centroid plus the largest |x - mu| per axis, without a second pass: rounding is
// monotonic, so max_i fl(|x_i - mu|) = max(fl(max_i x_i - mu), fl(mu - min_i x_i)) exactly.
__device__ __forceinline__ void model_centroid_absmax(const float *__restrict__ x, int L, int lane, float mu[3],
                                                      float mx[3], bool *finite)
{
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    bool ok = true;
#pragma unroll 4
    for (int i = lane; i < L; i += 32) {
        const float v0 = x[3 * i + 0], v1 = x[3 * i + 1], v2 = x[3 * i + 2];
        ok = ok && isfinite(v0) && isfinite(v1) && isfinite(v2);
        s0 += v0;
        s1 += v1;
        s2 += v2;
        lo[0] = fminf(lo[0], v0);
        lo[1] = fminf(lo[1], v1);
        lo[2] = fminf(lo[2], v2);
        hi[0] = fmaxf(hi[0], v0);
        hi[1] = fmaxf(hi[1], v1);
        hi[2] = fmaxf(hi[2], v2);
    }
    const double invL = 1.0 / (double)L;
    mu[0] = (float)(warp_sum_d((double)s0) * invL);
    mu[1] = (float)(warp_sum_d((double)s1) * invL);
    mu[2] = (float)(warp_sum_d((double)s2) * invL);
    *finite = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float l = -warp_max_f(-lo[ax]), h = warp_max_f(hi[ax]);
        mx[ax] = fmaxf(fmaxf(h - mu[ax], mu[ax] - l), 0.f);
    }
}

// FP32-SIMT layout. Grid: ceil(Npad/8) blocks of 256 threads (8 warps = 8 model slots).
__global__ void __launch_bounds__(256) prepass_simt_kernel(const float *__restrict__ coords, int64_t N, int L, int Lp,
                                                           int64_t Npad, float *__restrict__ Xk,
                                                           double *__restrict__ G64)
{
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (a >= Npad) return;
    if (a >= N) {
        for (int i = lane; i < Lp; i += 32)
            for (int ax = 0; ax < 3; ++ax) Xk[((int64_t)i * Npad + a) * 3 + ax] = 0.f;
        if (lane == 0) G64[a] = 0.0;
        return;
    }
    const float *x = coords + a * (int64_t)L * 3;
    float mu[3];
    bool finite;
    model_centroid(x, L, lane, mu, &finite);
    double g = 0.0;
    for (int i = lane; i < Lp; i += 32) {
        for (int ax = 0; ax < 3; ++ax) {
            float v = 0.f;
            if (i < L) v = x[3 * i + ax] - mu[ax];
            g += (double)v * (double)v;
            Xk[((int64_t)i * Npad + a) * 3 + ax] = v;
        }
    }
    g = warp_sum_d(g);
    if (lane == 0) {
        G64[a] = finite ? g : __longlong_as_double(0x7ff8000000000000ll);
        if (!finite) set_status(CLUSCO_ST_NONFINITE);
    }
}

// Exact-integer SIMT layout (see the header). Grid: ceil(Npad/8) blocks of 256 threads.
__global__ void __launch_bounds__(256) prepass_int_kernel(const float *__restrict__ coords, int64_t N, int L, int Lp,
                                                          int64_t Npad, int *__restrict__ Xn,
                                                          float *__restrict__ scales, double *__restrict__ G64)
{
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (a >= Npad) return;
    if (a >= N) {
        for (int i = lane; i < Lp; i += 32)
            for (int ax = 0; ax < 3; ++ax) Xn[((int64_t)i * Npad + a) * 3 + ax] = 0;
        if (lane < 3) scales[a * 3 + lane] = 1.f;
        if (lane == 0) G64[a] = 0.0;
        return;
    }
    const float *x = coords + a * (int64_t)L * 3;
    float mu[3], mx[3];
    bool finite;
    model_centroid_absmax(x, L, lane, mu, mx, &finite);
    float sc[3], inv[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const bool pos = mx[ax] > 0.f && isfinite(mx[ax]);
        sc[ax] = pos ? mx[ax] / Q24 : 1.f;
        inv[ax] = pos ? Q24 / mx[ax] : 1.f;
    }
    long long gi[3] = {0, 0, 0};
    for (int i = lane; i < Lp; i += 32) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            int ni = 0;
            if (i < L) {
                float n = rintf((x[3 * i + ax] - mu[ax]) * inv[ax]);
                n = isfinite(n) ? fminf(fmaxf(n, -Q24), Q24) : 0.f;
                ni = (int)n;
            }
            Xn[((int64_t)i * Npad + a) * 3 + ax] = ni;
            gi[ax] += (long long)ni * ni;
        }
    }
    double g = 0.0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) g += (double)sc[ax] * (double)sc[ax] * (double)warp_sum_ll(gi[ax]);
    if (lane < 3) scales[a * 3 + lane] = sc[lane];
    if (lane == 0) {
        G64[a] = finite ? g : __longlong_as_double(0x7ff8000000000000ll);
        if (!finite) set_status(CLUSCO_ST_NONFINITE);
    }
}

enum TcLayout { TC_EXACT2 = 0, TC_BF16X3 = 1, TC_TF32 = 2 };

// tcgen05 operand planes. Grid: ceil(Npad40/8) blocks of 256 threads.
// planes: element type bf16 (EXACT2, BF16X3; two planes) or float (TF32; one plane),
// plane stride Rpad*Lp elements. hplane / lplane (EXACT2, optional): the same 16-bit
// fixed-point coordinates as signed bytes, n = 256 h + l with h = floor((n + 128) / 256) and
// l = n - 256 h, both in [-128, 127] for |n| <= 32639, for the exact recomputation of flagged
// pairs with signed 4-way byte dot products.
template <int LAYOUT>
__global__ void __launch_bounds__(256) prepass_tc_kernel(const float *__restrict__ coords, int64_t N, int L, int Lp,
                                                         int64_t Npad, int64_t Rpad, void *__restrict__ planes,
                                                         float *__restrict__ scales, double *__restrict__ G64,
                                                         float *__restrict__ G32, float *__restrict__ xf,
                                                         int8_t *__restrict__ hplane = nullptr,
                                                         int8_t *__restrict__ lplane = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (a >= Npad) return;
    __nv_bfloat16 *p0 = reinterpret_cast<__nv_bfloat16 *>(planes);
    __nv_bfloat16 *p1 = p0 + Rpad * Lp;
    float *pf = reinterpret_cast<float *>(planes);
    const int64_t r0 = tc_row(a, 0);

    auto zero_row = [&](int64_t r) {
        for (int i = lane; i < Lp; i += 32) {
            if (LAYOUT == TC_TF32) {
                pf[r * Lp + i] = 0.f;
            } else {
                p0[r * Lp + i] = __float2bfloat16_rn(0.f);
                p1[r * Lp + i] = __float2bfloat16_rn(0.f);
            }
            if (xf) xf[r * Lp + i] = 0.f;
            if (hplane) {
                hplane[r * Lp + i] = 0;
                lplane[r * Lp + i] = 0;
            }
        }
    };
    if (a % 10 == 9) {  // the two padding rows that close this model's 32-row group
        zero_row(32 * (a / 10) + 30);
        zero_row(32 * (a / 10) + 31);
    }
    if (a >= N) {
        for (int ax = 0; ax < 3; ++ax) zero_row(r0 + ax);
        if (lane < 3) scales[a * 3 + lane] = 1.f;
        if (lane == 0) {
            G64[a] = 0.0;
            G32[a] = 0.f;
        }
        return;
    }
    const float *x = coords + a * (int64_t)L * 3;
    float mu[3], mx[3];
    bool finite;
    if (LAYOUT == TC_EXACT2)
        model_centroid_absmax(x, L, lane, mu, mx, &finite);
    else
        model_centroid(x, L, lane, mu, &finite);

    float inv[3] = {1.f, 1.f, 1.f}, sc[3] = {1.f, 1.f, 1.f};
    if (LAYOUT == TC_EXACT2) {
        for (int ax = 0; ax < 3; ++ax) {
            if (mx[ax] > 0.f && isfinite(mx[ax])) {
                sc[ax] = mx[ax] / 32639.f;
                inv[ax] = 32639.f / mx[ax];
            }
        }
    }
    long long gi[3] = {0, 0, 0};
    double gd = 0.0;
#pragma unroll 4
    for (int i = lane; i < Lp; i += 32) {
        for (int ax = 0; ax < 3; ++ax) {
            const int64_t off = (r0 + ax) * Lp + i;
            const float v = (i < L) ? (x[3 * i + ax] - mu[ax]) : 0.f;
            if (xf) xf[off] = v;
            if (LAYOUT == TC_EXACT2) {
                float n = rintf(v * inv[ax]);
                n = fminf(fmaxf(n, -32639.f), 32639.f);
                if (!isfinite(v)) n = 0.f;
                const float h = rintf(n * (1.f / 256.f));
                const float l = n - 256.f * h;
                p0[off] = __float2bfloat16_rn(h);
                p1[off] = __float2bfloat16_rn(l);
                const int ni = (int)n;
                if (hplane) {
                    const int hb = (ni + 128) >> 8;  // floor: n = 256 h + l, h and l in [-128, 127]
                    hplane[off] = (int8_t)hb;
                    lplane[off] = (int8_t)(ni - 256 * hb);
                }
                gi[ax] += (long long)ni * ni;
            } else if (LAYOUT == TC_BF16X3) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
                p0[off] = h;
                p1[off] = l;
                const double w = (double)__bfloat162float(h) + (double)__bfloat162float(l);
                gd += w * w;
            } else {
                uint32_t t;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
                const float tv = __uint_as_float(t);
                pf[off] = tv;
                gd += (double)tv * (double)tv;
            }
        }
    }
    double g;
    if (LAYOUT == TC_EXACT2) {
        g = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            const long long s = warp_sum_ll(gi[ax]);
            g += (double)sc[ax] * (double)sc[ax] * (double)s;
        }
    } else {
        g = warp_sum_d(gd);
    }
    if (lane < 3) scales[a * 3 + lane] = sc[lane];
    if (lane == 0) {
        if (!finite) {
            g = __longlong_as_double(0x7ff8000000000000ll);
            set_status(CLUSCO_ST_NONFINITE);
        }
        G64[a] = g;
        G32[a] = (float)g;
    }
}

}  // namespace clusco

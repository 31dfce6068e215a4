// vsref.cuh -- one-versus-reference cRMSD (every model against one reference model).
//
// HBM-bound: each model's 12 L bytes are streamed once (one warp per model, three passes
// that hit L1). The covariance is exact: centred coordinates are rounded to 24-bit fixed
// point per model and axis (step max|x| / (2^23 - 1)), the 9 products and 3 squares are
// accumulated in int64 (|n| < 2^23, so L < 2^17 cannot overflow), and the FP64 epilogue
// (an FP32 start polished by FP64 Newton on the quartic) turns them into cRMSD.
#pragma once
#include "common.cuh"
#include "epilogue.cuh"
#include "prepass.cuh"

namespace clusco {

struct RefInfo {
    float scale[3];
    float mu[3];
    double G;
    int finite;
};

// One block of RP_THREADS threads quantises the reference: nref[i][axis] (int32). Eight warps
// keep the FP64 block reductions (centroid, G) short: the FP64 pipe is 1/64 of FP32 here.
constexpr int RP_THREADS = 256;
constexpr int RP_WARPS = RP_THREADS / 32;

__global__ void __launch_bounds__(RP_THREADS) ref_prepass_kernel(const float *__restrict__ ref, int L,
                                                                 int *__restrict__ nref, RefInfo *__restrict__ info)
{
    __shared__ double red[RP_WARPS][3];
    __shared__ float mx[RP_WARPS][3];
    __shared__ long long gred[RP_WARPS][3];
    __shared__ int bad;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    double s[3] = {0, 0, 0};
    bool ok = true;
    for (int i = threadIdx.x; i < L; i += RP_THREADS)
        for (int ax = 0; ax < 3; ++ax) {
            const float v = ref[3 * i + ax];
            ok = ok && isfinite(v);
            s[ax] += (double)v;
        }
    __syncthreads();
    if (!ok) atomicOr(&bad, 1);
    for (int ax = 0; ax < 3; ++ax) {
        const double t = warp_sum_d(s[ax]);
        if (lane == 0) red[w][ax] = t;
    }
    __syncthreads();
    float mu[3];
    for (int ax = 0; ax < 3; ++ax) {
        double t = 0;
        for (int k = 0; k < RP_WARPS; ++k) t += red[k][ax];
        mu[ax] = (float)(t / (double)L);
    }
    float m[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < L; i += RP_THREADS)
        for (int ax = 0; ax < 3; ++ax) m[ax] = fmaxf(m[ax], fabsf(ref[3 * i + ax] - mu[ax]));
    for (int ax = 0; ax < 3; ++ax) {
        const float t = warp_max_f(m[ax]);
        if (lane == 0) mx[w][ax] = t;
    }
    __syncthreads();
    float sc[3], inv[3];
    for (int ax = 0; ax < 3; ++ax) {
        float t = 0.f;
        for (int k = 0; k < RP_WARPS; ++k) t = fmaxf(t, mx[k][ax]);
        sc[ax] = (t > 0.f && isfinite(t)) ? t / Q24 : 1.f;
        inv[ax] = (t > 0.f && isfinite(t)) ? Q24 / t : 1.f;
    }
    long long g[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < L; i += RP_THREADS)
        for (int ax = 0; ax < 3; ++ax) {
            const float v = ref[3 * i + ax] - mu[ax];
            float n = rintf(v * inv[ax]);
            n = isfinite(n) ? fminf(fmaxf(n, -Q24), Q24) : 0.f;
            const int ni = (int)n;
            nref[3 * i + ax] = ni;
            g[ax] += (long long)ni * ni;
        }
    for (int ax = 0; ax < 3; ++ax) {
        const long long t = warp_sum_ll(g[ax]);
        if (lane == 0) gred[w][ax] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double G = 0;
        for (int ax = 0; ax < 3; ++ax) {
            long long t = 0;
            for (int k = 0; k < RP_WARPS; ++k) t += gred[k][ax];
            G += (double)sc[ax] * (double)sc[ax] * (double)t;
            info->scale[ax] = sc[ax];
            info->mu[ax] = mu[ax];
        }
        info->G = G;
        info->finite = bad ? 0 : 1;
        if (bad) set_status(CLUSCO_ST_NONFINITE);
    }
}

// A block of 8 warps scores 8 models: each warp reduces the exact integer sums of one model
// (reference staged in dynamic shared memory, 12 L bytes), then warp 0 runs the 8 FP64
// epilogues side by side, one model per lane. (With 32 models per block, four per warp, the
// grid was about one block per SM and the integer sums' load latency dominated.)
constexpr int VSREF_MODELS = 8;

__global__ void __launch_bounds__(256) vsref_kernel(const float *__restrict__ coords, int64_t N, int L,
                                                    const int *__restrict__ nref_g, const RefInfo *__restrict__ info,
                                                    float *__restrict__ out)
{
    extern __shared__ int nref[];
    __shared__ long long sh[VSREF_MODELS][9];
    __shared__ long long sg[VSREF_MODELS][3];
    __shared__ float ssc[VSREF_MODELS][3];
    __shared__ int sfin[VSREF_MODELS];
    for (int i = threadIdx.x; i < 3 * L; i += blockDim.x) nref[i] = nref_g[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m0 = (int64_t)blockIdx.x * VSREF_MODELS;
    for (int mm = warp; mm < VSREF_MODELS; mm += 8) {
        const int64_t a = m0 + mm;
        if (a >= N) break;
        const float *x = coords + a * (int64_t)L * 3;
        float mu[3], mx[3];
        bool finite;
        model_centroid_absmax(x, L, lane, mu, mx, &finite);
        float inv[3], sc[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const bool pos = mx[ax] > 0.f && isfinite(mx[ax]);
            sc[ax] = pos ? mx[ax] / Q24 : 1.f;
            inv[ax] = pos ? Q24 / mx[ax] : 1.f;
        }
        long long h[9], g[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) h[k] = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) g[k] = 0;
        for (int i = lane; i < L; i += 32) {
            int n[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                float v = rintf((x[3 * i + ax] - mu[ax]) * inv[ax]);
                v = isfinite(v) ? fminf(fmaxf(v, -Q24), Q24) : 0.f;
                n[ax] = (int)v;
                g[ax] += (long long)n[ax] * n[ax];
            }
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) h[3 * al + be] += (long long)n[al] * nref[3 * i + be];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) h[k] = warp_sum_ll(h[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) g[k] = warp_sum_ll(g[k]);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 9; ++k) sh[mm][k] = h[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                sg[mm][k] = g[k];
                ssc[mm][k] = sc[k];
            }
            sfin[mm] = finite ? 1 : 0;
        }
    }
    __syncthreads();
    if (warp == 0 && lane < VSREF_MODELS) {
        const int64_t a = m0 + lane;
        if (a < N) {
            const RefInfo ri = *info;
            double H[9];
            double Ga = 0.0;
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const double sa = (double)ssc[lane][al];
                Ga += sa * sa * (double)sg[lane][al];
#pragma unroll
                for (int be = 0; be < 3; ++be) H[3 * al + be] = (sa * (double)ri.scale[be]) * (double)sh[lane][3 * al + be];
            }
            float c;
            if (!sfin[lane] || !ri.finite) {
                c = __int_as_float(0x7fc00000);
                if (!sfin[lane]) set_status(CLUSCO_ST_NONFINITE);
            } else {
                // FP32 start (cubic + two Newton steps on the normalised covariance), then FP64
                // Newton on the exact covariance: no FP64 trigonometry unless the root is degenerate
                const double Gs = Ga + ri.G;
                const double nrm = Gs > 0.0 ? 2.0 / Gs : 0.0;
                float mf[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) mf[k] = (float)(H[k] * nrm);
                c = crmsd_refine_newton_fp64(H, Ga, ri.G, 1.0 / (double)L, sigma_hat_f32(mf));
            }
            out[a] = c;
        }
    }
}

}  // namespace clusco

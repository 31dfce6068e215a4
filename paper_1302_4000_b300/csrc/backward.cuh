// backward.cuh -- adjoint of the all-pairs cRMSD matrix for a weighted loss.
//
// For Loss = sum_{a<b} w_ab c_ab (w = grad_out), the envelope theorem (R and t optimal)
// gives dc_ab/da_i = (a_i - R_ab b_i) / (L c_ab), R_ab the rotation superposing centred b
// onto centred a; centring is a projection whose chain rule is a no-op on residuals that
// sum to zero (it is applied anyway). With w~_ab = w_ab / (L max(c_ab, eps)):
//     g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,
// a contraction of the 3N x 3N block matrix of w~ R with the 3N x L coordinates.
//
// Rotations are recomputed here, never stored. Each CTA owns 32 models (rows) and sweeps
// all 32-model column tiles: FP32 CUDA-core covariance of the tile, per-pair rotation
// (FP32, dSigma/dM; Horn's adjugate near a double root, Jacobi sweeps where that is degenerate)
// scaled by w~ into
// shared memory, then the contraction into the row
// block's gradient (kept in the workspace; the row block is owned by one CTA, so there
// are no atomics). Pairs with c below CLUSCO_NEARDUP (A) are left out of that path: the
// GEMM form a - R b cancels like |x|/c there, so they are queued and handled by a direct
// FP64 residual kernel (recentred from the FP32 input, FP64 covariance, Horn rotation with a
// Newton-polished eigenvalue, Jacobi sweeps where the top eigenvalue is repeated, c
// recomputed from the residuals).
#pragma once
#include "common.cuh"
#include "epilogue.cuh"
#include "prepass.cuh"
#include "rotation.cuh"

#ifndef CLUSCO_NEARDUP
#define CLUSCO_NEARDUP 0.5f
#endif

namespace clusco {

constexpr int BW_T = 32;    // models per backward tile side
constexpr int BW_KC = 16;   // atoms per covariance K chunk
constexpr int BW_AB = 32;   // atoms per contraction block
constexpr size_t BW_SMEM = sizeof(float) * (2 * BW_KC * BW_T * 3 + BW_T * BW_T * 12 + BW_T * 3 * BW_AB + BW_T);

struct BwWs {
    float *Xk = nullptr;        // [Lp][Npad][3] centred FP32 (prepass_simt layout)
    double *G64 = nullptr;      // [Npad]
    float *Gacc = nullptr;      // [Npad][Lp][3] gradient accumulator
    long long *nd_list = nullptr;
    unsigned long long *nd_count = nullptr;
    int64_t Lp = 0, Npad = 0, nd_cap = 0;
    size_t bytes = 0;
};

inline BwWs carve_bw(void *base, int64_t N, int64_t L)
{
    BwWs w;
    size_t off = 0;
    char *b = (char *)base;
    auto take = [&](size_t n) {
        void *p = b ? b + off : nullptr;
        off = (off + n + 255) & ~size_t(255);
        return p;
    };
    w.Lp = (L + BW_KC - 1) / BW_KC * BW_KC;
    w.Lp = (w.Lp + BW_AB - 1) / BW_AB * BW_AB;
    w.Npad = (N + SIMT_TILE - 1) / SIMT_TILE * SIMT_TILE;
    w.Xk = (float *)take(sizeof(float) * w.Lp * w.Npad * 3);
    w.G64 = (double *)take(sizeof(double) * w.Npad);
    w.Gacc = (float *)take(sizeof(float) * w.Npad * w.Lp * 3);
    const int64_t P = N * (N - 1) / 2;
    w.nd_cap = nd_cap_for(P);
    w.nd_list = (long long *)take(sizeof(long long) * 2 * w.nd_cap);
    w.nd_count = (unsigned long long *)take(sizeof(unsigned long long));
    w.bytes = off;
    return w;
}

inline size_t backward_simt_ws_bytes(int64_t N, int64_t L) { return carve_bw(nullptr, N, L).bytes; }

// grid: Npad/32 CTAs of 256 threads.
__global__ void __launch_bounds__(256, 1)
    bwd_main_kernel(const float *__restrict__ Xk, const double *__restrict__ G64, int64_t N, int64_t Npad, int Lp,
                    int L, const float *__restrict__ wvec, const float *__restrict__ crmsd, float eps,
                    float *__restrict__ Gacc, float *__restrict__ grad, long long *__restrict__ nd_list,
                    unsigned long long *__restrict__ nd_count, int64_t nd_cap)
{
    extern __shared__ __align__(16) float bw_smem[];
    float(*As)[BW_T * 3] = reinterpret_cast<float(*)[BW_T * 3]>(bw_smem);
    float(*Bs)[BW_T * 3] = reinterpret_cast<float(*)[BW_T * 3]>(bw_smem + BW_KC * BW_T * 3);
    float(*Ps)[BW_T][12] = reinterpret_cast<float(*)[BW_T][12]>(bw_smem + 2 * BW_KC * BW_T * 3);  // w~ R_ab
    float(*Xs)[3][BW_AB] = reinterpret_cast<float(*)[3][BW_AB]>(bw_smem + 2 * BW_KC * BW_T * 3 + BW_T * BW_T * 12);
    float *dsum = bw_smem + 2 * BW_KC * BW_T * 3 + BW_T * BW_T * 12 + BW_T * 3 * BW_AB;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t I = blockIdx.x;
    const int64_t a0 = I * BW_T;
    const int64_t T = Npad / BW_T;
    const float invL = 1.f / (float)L;
    if (tid < BW_T) dsum[tid] = 0.f;
    // zero this row block's accumulator
    for (int64_t e = tid; e < (int64_t)BW_T * Lp * 3; e += 256) Gacc[a0 * Lp * 3 + e] = 0.f;
    __syncthreads();

    for (int64_t J = 0; J < T; ++J) {
        const int64_t b0 = J * BW_T;
        if (b0 >= N) break;
        // (1) covariance of the 32 x 32 tile: thread owns A-models 2ty+{0,1}, B-models 2tx+{0,1}
        float acc[2][2][9];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 9; ++e) acc[i][j][e] = 0.f;
        for (int k0 = 0; k0 < Lp; k0 += BW_KC) {
            for (int v = tid; v < 2 * BW_KC * 24; v += 256) {
                const int which = v / (BW_KC * 24), rem = v % (BW_KC * 24);
                const int k = rem / 24, q = rem % 24;
                const int64_t base = which ? b0 : a0;
                const float4 val = *reinterpret_cast<const float4 *>(Xk + ((int64_t)(k0 + k) * Npad + base) * 3 + 4 * q);
                *reinterpret_cast<float4 *>(which ? &Bs[k][4 * q] : &As[k][4 * q]) = val;
            }
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < BW_KC; ++k) {
                float av[6], bv[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    av[q] = As[k][ty * 6 + q];
                    bv[q] = Bs[k][tx * 6 + q];
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int al = 0; al < 3; ++al)
#pragma unroll
                            for (int be = 0; be < 3; ++be)
                                acc[i][j][3 * al + be] = fmaf(av[3 * i + al], bv[3 * j + be], acc[i][j][3 * al + be]);
            }
            __syncthreads();
        }
        // (2) per pair: w~ R_ab into Ps (zero for masked and near-duplicate pairs)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int la = 2 * ty + i, lb = 2 * tx + j;
                const int64_t a = a0 + la, b = b0 + lb;
                float P[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                float coef = 0.f;
                if (a < N && b < N && a != b) {
                    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
                    const int64_t idx = condensed_idx(lo, hi, N);
                    const float c = crmsd[idx];
                    const float w = wvec[idx];
                    if (!(c >= CLUSCO_NEARDUP)) {
                        if (a < b && w != 0.f) {
                            const unsigned long long slot = atomicAdd(nd_count, 1ull);
                            if ((int64_t)slot < nd_cap) {
                                nd_list[2 * slot] = a;
                                nd_list[2 * slot + 1] = b;
                            }
                        }
                    } else if (w != 0.f) {
                        const float Ga = (float)G64[a], Gb = (float)G64[b];
                        float s, errc2;
                        crmsd_fast_fp32(acc[i][j], Ga, Gb, invL, &s, &errc2);
                        const float nrm = 2.f / (Ga + Gb);
                        float Hn[9];
#pragma unroll
                        for (int e = 0; e < 9; ++e) Hn[e] = acc[i][j][e] * nrm;
                        float R[9];
                        if (!rotation_from_sigma_f32(Hn, s, R) && !horn_rotation(Hn, s, 1e-5f, R))
                            rotation_jacobi4<float, 8>(Hn, R);
                        coef = w / ((float)L * fmaxf(c, eps));
#pragma unroll
                        for (int e = 0; e < 9; ++e) P[e] = coef * R[e];
                    }
                }
#pragma unroll
                for (int e = 0; e < 9; ++e) Ps[la][lb][e] = P[e];
                if (coef != 0.f) atomicAdd(&dsum[la], coef);
            }
        }
        __syncthreads();
        // (3) contraction: Gacc[a][i] -= sum_b P_ab x_b,i. thread = (a-group of 4, atom lane)
        const int ag = tid >> 5, il = tid & 31;
        for (int i0 = 0; i0 < Lp; i0 += BW_AB) {
            for (int v = tid; v < BW_T * 3 * BW_AB; v += 256) {
                const int lb = v / (3 * BW_AB), rem = v % (3 * BW_AB);
                const int ax = rem / BW_AB, ii = rem % BW_AB;
                Xs[lb][ax][ii] = Xk[((int64_t)(i0 + ii) * Npad + b0 + lb) * 3 + ax];
            }
            __syncthreads();
            float g[4][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q][0] = g[q][1] = g[q][2] = 0.f;
            for (int lb = 0; lb < BW_T; ++lb) {
                const float x0 = Xs[lb][0][il], x1 = Xs[lb][1][il], x2 = Xs[lb][2][il];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float *p = Ps[4 * ag + q][lb];
                    g[q][0] += p[0] * x0 + p[1] * x1 + p[2] * x2;
                    g[q][1] += p[3] * x0 + p[4] * x1 + p[5] * x2;
                    g[q][2] += p[6] * x0 + p[7] * x1 + p[8] * x2;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float *dst = Gacc + ((a0 + 4 * ag + q) * Lp + i0 + il) * 3;
                dst[0] -= g[q][0];
                dst[1] -= g[q][1];
                dst[2] -= g[q][2];
            }
            __syncthreads();
        }
    }
    // (4) finish: g_a = dsum_a * x_a + Gacc_a, minus its mean over atoms (centring chain rule)
    const int w = tid >> 5, lane = tid & 31;
    for (int la = w; la < BW_T; la += 8) {
        const int64_t a = a0 + la;
        if (a >= N) continue;
        const float d = dsum[la];
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
        for (int i = lane; i < L; i += 32) {
            const float *ga = Gacc + (a * Lp + i) * 3;
            m0 += ga[0] + d * Xk[((int64_t)i * Npad + a) * 3 + 0];
            m1 += ga[1] + d * Xk[((int64_t)i * Npad + a) * 3 + 1];
            m2 += ga[2] + d * Xk[((int64_t)i * Npad + a) * 3 + 2];
        }
        m0 = warp_sum_f(m0) / (float)L;
        m1 = warp_sum_f(m1) / (float)L;
        m2 = warp_sum_f(m2) / (float)L;
        for (int i = lane; i < L; i += 32) {
            const float *ga = Gacc + (a * Lp + i) * 3;
            float *out = grad + (a * (int64_t)L + i) * 3;
            out[0] = ga[0] + d * Xk[((int64_t)i * Npad + a) * 3 + 0] - m0;
            out[1] = ga[1] + d * Xk[((int64_t)i * Npad + a) * 3 + 1] - m1;
            out[2] = ga[2] + d * Xk[((int64_t)i * Npad + a) * 3 + 2] - m2;
        }
    }
}

// Direct FP64 path for near-duplicate pairs: one warp per queued pair (a < b), pairs spread
// over the blocks first (so over the SMs). Centroids from per-lane compensated FP32 sums
// (Neumaier: a running error term, so each lane's sum is exact to a few units of FP32
// rounding squared) combined in FP64; the centred coordinates, G_A, G_B and the covariance in
// FP64; the
// rotation in FP64 (quartic Newton, Horn's adjugate, Jacobi where that vanishes); cRMSD from
// L c^2 = G_A + G_B - 2 tr(R^T H) in FP64 (stationary in R, and the cancellation leaves ~1e-12
// relative of G at FP64 rounding); then one more pass for the residuals a_i - R b_i in FP64
// and the gradient terms: the b side b_i - R^T a_i = -R^T (a_i - R b_i) from the FP64
// residual rounded to FP32 (accurate relative to the residual itself).
__global__ void __launch_bounds__(256, 2) bwd_neardup_kernel(const float *__restrict__ coords, int64_t N, int L,
                                                          const float *__restrict__ wvec, float eps,
                                                          const long long *__restrict__ nd_list,
                                                          const unsigned long long *__restrict__ nd_count,
                                                          int64_t nd_cap, float *__restrict__ grad)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    unsigned long long cnt = *nd_count;
    if (cnt > (unsigned long long)nd_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(CLUSCO_ST_BOUNDS);
        cnt = nd_cap;
    }
    for (int64_t p = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; p < (int64_t)cnt; p += nwarps) {
        const int64_t a = nd_list[2 * p], b = nd_list[2 * p + 1];
        const float *xa = coords + a * (int64_t)L * 3;
        const float *xb = coords + b * (int64_t)L * 3;
        float fa[3] = {0.f, 0.f, 0.f}, fb[3] = {0.f, 0.f, 0.f}, ca[3] = {0.f, 0.f, 0.f}, cb[3] = {0.f, 0.f, 0.f};
        auto acc = [](float &sum, float &comp, float x) {
            const float t = sum + x;
            comp += fabsf(sum) >= fabsf(x) ? (sum - t) + x : (x - t) + sum;
            sum = t;
        };
        for (int i = lane; i < L; i += 32)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                acc(fa[k], ca[k], xa[3 * i + k]);
                acc(fb[k], cb[k], xb[3 * i + k]);
            }
        double ma[3], mb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ma[k] = warp_sum_d((double)fa[k] + (double)ca[k]) / (double)L;
            mb[k] = warp_sum_d((double)fb[k] + (double)cb[k]) / (double)L;
        }
        double H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, Ga = 0, Gb = 0;
        for (int i = lane; i < L; i += 32) {
            double u[3], v[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                u[k] = (double)xa[3 * i + k] - ma[k];
                v[k] = (double)xb[3 * i + k] - mb[k];
                Ga = fma(u[k], u[k], Ga);
                Gb = fma(v[k], v[k], Gb);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) H[3 * r + c] = fma(u[r], v[c], H[3 * r + c]);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) H[k] = warp_sum_d(H[k]);
        Ga = warp_sum_d(Ga);
        Gb = warp_sum_d(Gb);
        const double Gs = Ga + Gb;
        double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (Gs > 0.0) {
            double m[9];
            const double nrm = 2.0 / Gs;
#pragma unroll
            for (int k = 0; k < 9; ++k) m[k] = H[k] * nrm;
            double I1, det, I2;
            invariants3(m, I1, det, I2);
            bool deg;
            double s = quartic_newton(sigma_cubic_d(I1, det, I2), I1, det, I2, 3, &deg);
            if (deg) s = sigma_cubic_d(I1, det, I2);
            if (!horn_rotation(m, s, 1e-12, R)) rotation_jacobi4<double, 10>(m, R);
        }
        double tr = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) tr = fma(R[k], H[k], tr);
        const double c = sqrt(fmax(Gs - 2.0 * tr, 0.0) / (double)L);
        const double w = (double)wvec[condensed_idx(a, b, N)];
        const float coef = (float)(w / ((double)L * fmax(c, (double)eps)));
        float Rf[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Rf[k] = (float)R[k];
        // a side: coef (a_i - R b_i); b side: coef (b_i - R^T a_i). Both sum to zero over atoms.
        // Added into the gradient with FP32 atomics (several queued pairs share a model): the
        // order of the additions, hence the last bits of the gradient rows of models with
        // near-duplicates, varies from run to run; each term is FP64-accurate before rounding,
        // so the run-to-run spread is a few FP32 ulps of the row, far below the 1e-3 relative
        // tolerance of the adjoint.
        for (int i = lane; i < L; i += 32) {
            double u[3], v[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                u[k] = (double)xa[3 * i + k] - ma[k];
                v[k] = (double)xb[3 * i + k] - mb[k];
            }
            float ea[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                ea[r] = (float)fma(-R[3 * r + 2], v[2], fma(-R[3 * r + 1], v[1], fma(-R[3 * r], v[0], u[r])));
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float eb = -fmaf(Rf[6 + r], ea[2], fmaf(Rf[3 + r], ea[1], Rf[r] * ea[0]));
                atomicAdd(grad + (a * (int64_t)L + i) * 3 + r, coef * ea[r]);
                atomicAdd(grad + (b * (int64_t)L + i) * 3 + r, coef * eb);
            }
        }
    }
}

inline int backward_simt_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                           float *grad, float eps, int form, void *ws, cudaStream_t st, std::string &err)
{
    (void)form;
    const BwWs w = carve_bw(ws, N, L);
    prepass_simt_kernel<<<(unsigned)((w.Npad + 7) / 8), 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Xk,
                                                                        w.G64);
    cudaError_t e = cudaMemsetAsync(w.nd_count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        e = cudaFuncSetAttribute(bwd_main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BW_SMEM);
    }
    if (e == cudaSuccess) {
        bwd_main_kernel<<<(unsigned)(w.Npad / BW_T), 256, BW_SMEM, st>>>(w.Xk, w.G64, N, w.Npad, (int)w.Lp, (int)L, grad_out,
                                                                   crmsd, eps, w.Gacc, grad, w.nd_list, w.nd_count,
                                                                   w.nd_cap);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bwd_neardup_kernel<<<296, 256, 0, st>>>(coords, N, (int)L, grad_out, eps, w.nd_list, w.nd_count, w.nd_cap,
                                                grad);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("backward launch: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

}  // namespace clusco

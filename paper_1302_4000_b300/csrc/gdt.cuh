// gdt.cuh -- GDT_TS, TM-score and MaxSub of every model against a reference (ClusCo, section
// "Algorithms", eq. 3 and eq. 4), each the maximum over the paper's superposition search:
// seeds are the contiguous fragments of 4, L/4, L/2 and L atoms; the model is superimposed on
// the reference by the optimal rotation and translation of a seed's atoms, scored, and then
// superimposed again on the atoms that came within 3.5 A, until that number repeats, fewer
// than 3 atoms qualify, or four refinements were made.
//
// Layout: one block per model, the model and the reference staged in shared memory in FP64;
// each warp runs 32 seeds side by side, one per lane, so that the 4x4 eigenproblem of every
// superposition (Horn's quaternion form, cyclic Jacobi sweeps) runs once per lane instead of
// redundantly across a warp. Every lane walks all L atoms in the same order (broadcast reads).
// The decisions that make the scores integers -- d < 1, 2, 4, 8 A and the 3.5 A selection --
// are taken in FP64 like the oracle's, so they agree with it except at exact ties; the TM and
// MaxSub terms 1 / (1 + (d / d0)^2) are summed in FP32. One pass over the atoms scores a
// superposition and accumulates the moments of the atoms it selects, which give the next fit.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "rotation.cuh"

namespace clusco {

constexpr int GT_WARPS = 8;
constexpr int GT_THREADS = 32 * GT_WARPS;
constexpr int GT_MAX_L = 1024;

// d0 of the TM-score, 1.24 (L - 15)^(1/3) - 1.8 A, not below 0.5 A
__host__ __device__ __forceinline__ double gt_d0(int L)
{
    const double d0 = 1.24 * cbrt((double)L - 15.0) - 1.8;
    return d0 > 0.5 ? d0 : 0.5;
}

// The seed lengths 4, L/4, L/2, L (below 3 or above L dropped, repeats taken once); returns
// their number, lens[] and the number of seeds of each (L - len + 1).
__device__ __forceinline__ int gt_lengths(int L, int (&lens)[4])
{
    const int cand[4] = {4, L / 4, L / 2, L};
    int n = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        bool ok = cand[c] >= 3 && cand[c] <= L;
        for (int d = 0; d < n; ++d) ok = ok && lens[d] != cand[c];
        if (ok) lens[n++] = cand[c];
    }
    return n;
}

// Moments of a set of atom pairs (a_i reference, b_i model): sums of a, b and a b^T, and the count.
struct GtMoments {
    double sa[3], sb[3], sab[9];
    int n;
};

__device__ __forceinline__ void gt_zero(GtMoments &m)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) m.sa[k] = m.sb[k] = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) m.sab[k] = 0.0;
    m.n = 0;
}

__device__ __forceinline__ void gt_add(GtMoments &m, const double *a, const double *b)
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        m.sa[r] += a[r];
        m.sb[r] += b[r];
#pragma unroll
        for (int c = 0; c < 3; ++c) m.sab[3 * r + c] = fma(a[r], b[c], m.sab[3 * r + c]);
    }
    ++m.n;
}

// The superposition R b + t ~ a of the moments' atoms: H = sum (a - abar)(b - bbar)^T, R from
// Horn's key matrix by Jacobi sweeps, t = abar - R bbar.
__device__ __forceinline__ void gt_fit(const GtMoments &m, double R[9], double t[3])
{
    const double inv = 1.0 / (double)m.n;
    double ma[3], mb[3], H[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ma[k] = m.sa[k] * inv;
        mb[k] = m.sb[k] * inv;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) H[3 * r + c] = m.sab[3 * r + c] - m.sa[r] * mb[c];
    rotation_jacobi4<double, 10>(H, R);
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = ma[r] - (R[3 * r] * mb[0] + R[3 * r + 1] * mb[1] + R[3 * r + 2] * mb[2]);
}

__global__ void __launch_bounds__(GT_THREADS) gdt_tm_kernel(const float *__restrict__ coords, int64_t N, int L,
                                                            const float *__restrict__ ref, float *__restrict__ out)
{
    extern __shared__ double gs[];  // reference a[L][3], then model b[L][3]
    __shared__ int wbest_c[GT_WARPS][4];
    __shared__ float wbest_f[GT_WARPS][2];
    double *sa = gs, *sb = gs + 3 * L;
    const int64_t m = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = true;
    for (int t = threadIdx.x; t < 3 * L; t += blockDim.x) {
        const float va = __ldg(ref + t), vb = __ldg(coords + m * (int64_t)L * 3 + t);
        ok = ok && isfinite(va) && isfinite(vb);
        sa[t] = (double)va;
        sb[t] = (double)vb;
    }
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
            out[3 * m] = out[3 * m + 1] = out[3 * m + 2] = __int_as_float(0x7fc00000);
            set_status(CLUSCO_ST_NONFINITE);
        }
        return;
    }
    int lens[4];
    const int nl = gt_lengths(L, lens);
    int S = 0;
    for (int c = 0; c < nl; ++c) S += L - lens[c] + 1;
    const double d0 = gt_d0(L);
    const float k_tm = (float)(1.0 / (d0 * d0)), k_ms = 1.f / 12.25f;

    int best_c[4] = {0, 0, 0, 0};
    float best_tm = 0.f, best_ms = 0.f;
    for (int s_base = 32 * warp; s_base < S; s_base += 32 * GT_WARPS) {
        // this lane's seed: fragment [s0, s0 + len)
        const int s = s_base + lane;
        bool active = s < S;
        int s0 = 0, len = 0;
        {
            int r = s;
            for (int c = 0; c < nl; ++c) {
                const int cnt = L - lens[c] + 1;
                if (r >= 0 && r < cnt) {
                    len = lens[c];
                    s0 = r;
                }
                r -= cnt;
            }
        }
        GtMoments mom;
        gt_zero(mom);
        if (active)
            for (int i = s0; i < s0 + len; ++i) gt_add(mom, sa + 3 * i, sb + 3 * i);
        int prev = -1;
        for (int it = 0; it <= 4 && __any_sync(0xffffffffu, active); ++it) {
            double R[9], t[3];
            if (active) gt_fit(mom, R, t);
            GtMoments next;
            gt_zero(next);
            int c[4] = {0, 0, 0, 0};
            float tm = 0.f, ms = 0.f;
            if (active) {
                for (int i = 0; i < L; ++i) {
                    const double *ai = sa + 3 * i, *bi = sb + 3 * i;
                    double d2 = 0.0;
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const double e = fma(R[3 * r], bi[0], fma(R[3 * r + 1], bi[1], fma(R[3 * r + 2], bi[2], t[r]))) - ai[r];
                        d2 = fma(e, e, d2);
                    }
                    c[0] += d2 < 1.0;
                    c[1] += d2 < 4.0;
                    c[2] += d2 < 16.0;
                    c[3] += d2 < 64.0;
                    const float df = (float)d2;
                    tm += __frcp_rn(fmaf(df, k_tm, 1.f));
                    ms += __frcp_rn(fmaf(df, k_ms, 1.f));
                    if (d2 < 12.25) gt_add(next, ai, bi);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) best_c[k] = max(best_c[k], c[k]);
                best_tm = fmaxf(best_tm, tm);
                best_ms = fmaxf(best_ms, ms);
                const int ns = next.n;
                if (it == 4 || ns < 3 || ns == prev) {
                    active = false;
                } else {
                    prev = ns;
                    mom = next;
                }
            }
        }
    }
    // maxima over the warp's lanes, then over the block's warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) best_c[k] = max(best_c[k], __shfl_xor_sync(0xffffffffu, best_c[k], o));
        best_tm = fmaxf(best_tm, __shfl_xor_sync(0xffffffffu, best_tm, o));
        best_ms = fmaxf(best_ms, __shfl_xor_sync(0xffffffffu, best_ms, o));
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) wbest_c[warp][k] = best_c[k];
        wbest_f[warp][0] = best_tm;
        wbest_f[warp][1] = best_ms;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cmax[4] = {0, 0, 0, 0};
        float tmax = 0.f, mmax = 0.f;
        for (int w = 0; w < GT_WARPS; ++w) {
            for (int k = 0; k < 4; ++k) cmax[k] = max(cmax[k], wbest_c[w][k]);
            tmax = fmaxf(tmax, wbest_f[w][0]);
            mmax = fmaxf(mmax, wbest_f[w][1]);
        }
        out[3 * m] = (float)((double)(cmax[0] + cmax[1] + cmax[2] + cmax[3]) / (4.0 * (double)L));
        out[3 * m + 1] = tmax / (float)L;
        out[3 * m + 2] = mmax / (float)L;
    }
}

inline int gdt_tm_launch(const float *coords, int64_t N, int64_t L, const float *ref, float *out, cudaStream_t st,
                         std::string &err)
{
    const size_t smem = (size_t)L * 6 * sizeof(double);
    cudaError_t e = cudaSuccess;
    // the static shared arrays count against the default 48 KB too, so the dynamic limit is raised
    // whenever the staged coordinates come near it
    if (smem > 40 * 1024) e = cudaFuncSetAttribute(gdt_tm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        gdt_tm_kernel<<<(unsigned)N, GT_THREADS, smem, st>>>(coords, N, (int)L, ref, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("gdt_tm_kernel: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

}  // namespace clusco

// gdt.cuh -- GDT_TS, TM-score and MaxSub of every model against a reference (ClusCo, section
// "Algorithms", eq. 3 and eq. 4), each the maximum over the paper's superposition search:
// seeds are the contiguous fragments of 4, L/4, L/2 and L atoms; the model is superimposed on
// the reference by the optimal rotation and translation of a seed's atoms, scored, and then
// superimposed again on the atoms that came within 3.5 A, until the number of selected atoms has
// not changed in four iterations (four refinements in a row select as many atoms as the one
// before), fewer than 3 atoms qualify, or 20 refinements were made; a refinement that selects
// exactly the atoms it was fitted on (equal moments) repeats itself from then on, so the search
// stops there as well, with the same maxima.
//
// Layout: one block of four warps per model (five blocks per SM, where the latency-bound search
// balances occupancy against the registers it spills), the model and the reference staged in shared
// memory (as given, and centred); each warp runs 32 seeds side by side, one per lane, so that the eigenproblem of
// every superposition runs once per lane instead of redundantly across a warp, and every lane
// walks all L atoms in the same order (broadcast reads). One pass over the atoms scores a
// superposition and accumulates the moments of the atoms it selects, which give the next fit.
//
// Precision (B300's FP64 rate is 1/64 of FP32, so FP64 is kept off the per-atom path): the
// moments (sums of a, b, a b^T over the selected atoms) are accumulated from the given FP32
// coordinates as double-float values (exact products by FMA, compensated sums; two accumulators
// per paired FP32 instruction), good to about 2^-48; the superposition is solved in FP64 from them (the largest root of the key matrix's
// quartic by Newton from an upper bound, the rotation from the adjugate of K - lambda I, cyclic
// Jacobi sweeps where that root is nearly repeated); each atom's squared distance is then taken
// in FP32 in the centred frame, and where it falls within its error bound of a cutoff
// (1, 2, 3.5, 4, 8 A) it is recomputed in FP64 from the given coordinates. So every integer
// decision is the one FP64 arithmetic takes, as in the oracle; the TM and MaxSub terms
// 1 / (1 + (d / d0)^2) are summed in FP32.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "rotation.cuh"

namespace clusco {

constexpr int GT_WARPS = 4;
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

// Double-float accumulators: hi + lo, with the rounding error of every addition carried in lo
// (Knuth's two-sum) and products split exactly by FMA, kept in pairs so that two accumulators
// advance per paired FP32 instruction (__fadd2_rn, __ffma2_rn: each half an IEEE operation,
// the same sequence per accumulator as one at a time). The _rn intrinsics keep the compiler
// from contracting the error terms away.
__device__ __forceinline__ float2 gt_neg2(float2 v) { return make_float2(-v.x, -v.y); }

__device__ __forceinline__ void df2_add(float2 &hi, float2 &lo, float2 v)
{
    const float2 t = __fadd2_rn(hi, v);
    const float2 bp = __fadd2_rn(t, gt_neg2(hi));
    const float2 err = __fadd2_rn(__fadd2_rn(hi, gt_neg2(__fadd2_rn(t, gt_neg2(bp)))), __fadd2_rn(v, gt_neg2(bp)));
    hi = t;
    lo = __fadd2_rn(lo, err);
}

__device__ __forceinline__ void df2_add_prod(float2 &hi, float2 &lo, float2 a, float2 b)
{
    const float2 p = __fmul2_rn(a, b);
    const float2 e = __ffma2_rn(a, b, gt_neg2(p));  // a b - p exactly, per half
    df2_add(hi, lo, p);
    lo = __fadd2_rn(lo, e);
}

// Moments of a set of atom pairs (a_i reference, b_i model, as given): sums of a (slots 0..2),
// b (3..5) and a b^T (6..14, row-major); slot k is half k % 2 of pair k / 2 (slot 15 unused).
struct GtMoments {
    float2 hi[8], lo[8];
    int n;
};

__device__ __forceinline__ double gt_slot(const GtMoments &m, int k)
{
    const float2 h = m.hi[k >> 1], l = m.lo[k >> 1];
    return (k & 1) ? (double)h.y + (double)l.y : (double)h.x + (double)l.x;
}

constexpr int GT_STABLE = 4;       // iterations without a change of the selected count that end a search
constexpr int GT_MAX_REFINE = 20;  // refinements at most

// Bitwise equal moments (the same atoms summed in the same order): the same fit follows.
__device__ __forceinline__ bool gt_equal(const GtMoments &x, const GtMoments &y)
{
    bool eq = x.n == y.n;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        eq = eq && __float_as_uint(x.hi[k].x) == __float_as_uint(y.hi[k].x) &&
             __float_as_uint(x.hi[k].y) == __float_as_uint(y.hi[k].y) &&
             __float_as_uint(x.lo[k].x) == __float_as_uint(y.lo[k].x) &&
             __float_as_uint(x.lo[k].y) == __float_as_uint(y.lo[k].y);
    return eq;
}

__device__ __forceinline__ void gt_zero(GtMoments &m)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) m.hi[k] = m.lo[k] = make_float2(0.f, 0.f);
    m.n = 0;
}

__device__ __forceinline__ void gt_add(GtMoments &m, const float4 &a, const float4 &b)
{
    df2_add(m.hi[0], m.lo[0], make_float2(a.x, a.y));
    df2_add(m.hi[1], m.lo[1], make_float2(a.z, b.x));
    df2_add(m.hi[2], m.lo[2], make_float2(b.y, b.z));
    df2_add_prod(m.hi[3], m.lo[3], make_float2(a.x, a.x), make_float2(b.x, b.y));
    df2_add_prod(m.hi[4], m.lo[4], make_float2(a.x, a.y), make_float2(b.z, b.x));
    df2_add_prod(m.hi[5], m.lo[5], make_float2(a.y, a.y), make_float2(b.y, b.z));
    df2_add_prod(m.hi[6], m.lo[6], make_float2(a.z, a.z), make_float2(b.x, b.y));
    df2_add_prod(m.hi[7], m.lo[7], make_float2(a.z, 0.f), make_float2(b.z, 0.f));
    ++m.n;
}

// The optimal rotation for H = sum (a - abar)(b - bbar)^T in FP64. Its quality is the largest
// eigenvalue lambda of Horn's key matrix K(H), the largest root of
//   P(x) = x^4 - 2 I1 x^2 - 8 det(H) x + (I1^2 - 4 I2)
// (I1 = |H|_F^2, I2 = sum of the squared 2x2 minors), found by Newton from the upper bound
// sqrt(3 I1), where P is increasing and convex; the rotation comes from the adjugate of
// K - lambda I, or from Jacobi sweeps where lambda is nearly repeated.
__device__ __forceinline__ void gt_rotation(const double H[9], double R[9])
{
    double I1 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) I1 = fma(H[k], H[k], I1);
    const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                       H[2] * (H[3] * H[7] - H[4] * H[6]);
    double I2 = 0.0;
#pragma unroll
    for (int r0 = 0; r0 < 2; ++r0)
#pragma unroll
        for (int r1 = r0 + 1; r1 < 3; ++r1)
#pragma unroll
            for (int c0 = 0; c0 < 2; ++c0)
#pragma unroll
                for (int c1 = c0 + 1; c1 < 3; ++c1) {
                    const double mn = H[3 * r0 + c0] * H[3 * r1 + c1] - H[3 * r0 + c1] * H[3 * r1 + c0];
                    I2 = fma(mn, mn, I2);
                }
    const double c0 = I1 * I1 - 4.0 * I2;
    double x = sqrt(3.0 * I1);
    for (int k = 0; k < 60; ++k) {
        const double x2 = x * x;
        const double p = fma(x2, x2 - 2.0 * I1, fma(-8.0 * det, x, c0));
        const double dp = 4.0 * x * (x2 - I1) - 8.0 * det;
        if (!(dp > 0.0)) break;
        const double step = p / dp;
        x -= step;
        if (!(fabs(step) > 1e-15 * x)) break;
    }
    if (!(I1 > 0.0) || !horn_rotation<double>(H, x, 1e-6, R)) rotation_jacobi4<double, 10>(H, R);
}

// The superposition R b + t ~ a of the moments' atoms.
__device__ __forceinline__ void gt_fit(const GtMoments &m, double R[9], double t[3])
{
    const double inv = 1.0 / (double)m.n;
    double sa[3], mb[3], H[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sa[k] = gt_slot(m, k);
        mb[k] = gt_slot(m, 3 + k) * inv;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) H[3 * r + c] = gt_slot(m, 6 + 3 * r + c) - sa[r] * mb[c];
    gt_rotation(H, R);
#pragma unroll
    for (int r = 0; r < 3; ++r)
        t[r] = sa[r] * inv - (R[3 * r] * mb[0] + R[3 * r + 1] * mb[1] + R[3 * r + 2] * mb[2]);
}

__global__ void __launch_bounds__(GT_THREADS, 5) gdt_tm_kernel(const float *__restrict__ coords, int64_t N, int L,
                                                            const float *__restrict__ ref, float *__restrict__ out)
{
    // reference and model as given (fa, fb) and centred on their centroids in FP32 (ca, cb)
    extern __shared__ float4 gsm[];
    float4 *fa = gsm, *fb = gsm + L, *ca = gsm + 2 * L, *cb = gsm + 3 * L;
    __shared__ int wbest_c[GT_WARPS][4];
    __shared__ float wbest_f[GT_WARPS][2];
    __shared__ float s_cen[6];
    __shared__ float s_red[GT_WARPS][7];
    // each lane's current superposition in FP64 (R row-major, then t), read only by the rare
    // re-check near a cutoff, so that the atom loop does not hold it in registers
    __shared__ double s_rt[GT_WARPS][12][32];
    const int64_t m = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = true;
    float part[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const float *pa = ref + 3 * i, *pb = coords + (m * (int64_t)L + i) * 3;
        const float4 va = make_float4(__ldg(pa), __ldg(pa + 1), __ldg(pa + 2), 0.f);
        const float4 vb = make_float4(__ldg(pb), __ldg(pb + 1), __ldg(pb + 2), 0.f);
        ok = ok && isfinite(va.x) && isfinite(va.y) && isfinite(va.z) && isfinite(vb.x) && isfinite(vb.y) &&
             isfinite(vb.z);
        fa[i] = va;
        fb[i] = vb;
        part[0] += va.x;
        part[1] += va.y;
        part[2] += va.z;
        part[3] += vb.x;
        part[4] += vb.y;
        part[5] += vb.z;
    }
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
            out[3 * m] = out[3 * m + 1] = out[3 * m + 2] = __int_as_float(0x7fc00000);
            set_status(CLUSCO_ST_NONFINITE);
        }
        return;
    }
    // centroids (any FP32 values serve: the centred copies are only the fast path's frame)
#pragma unroll
    for (int k = 0; k < 6; ++k) part[k] = warp_sum_f(part[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) s_red[warp][k] = part[k];
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = 0.f;
        for (int w = 0; w < GT_WARPS; ++w) v += s_red[w][threadIdx.x];
        s_cen[threadIdx.x] = v / (float)L;
    }
    __syncthreads();
    const float cax = s_cen[0], cay = s_cen[1], caz = s_cen[2], cbx = s_cen[3], cby = s_cen[4], cbz = s_cen[5];
    float mc = 0.f;  // largest centred coordinate
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const float4 va = fa[i], vb = fb[i];
        const float4 a2 = make_float4(va.x - cax, va.y - cay, va.z - caz, 0.f);
        const float4 b2 = make_float4(vb.x - cbx, vb.y - cby, vb.z - cbz, 0.f);
        ca[i] = a2;
        cb[i] = b2;
        mc = fmaxf(mc, fmaxf(fmaxf(fabsf(a2.x), fabsf(a2.y)), fmaxf(fabsf(a2.z), fmaxf(fabsf(b2.x), fmaxf(fabsf(b2.y), fabsf(b2.z))))));
    }
    mc = warp_max_f(mc);
    if (lane == 0) s_red[warp][6] = mc;
    __syncthreads();
    mc = 0.f;
    for (int w = 0; w < GT_WARPS; ++w) mc = fmaxf(mc, s_red[w][6]);

    int lens[4];
    const int nl = gt_lengths(L, lens);
    int S = 0;
    for (int c = 0; c < nl; ++c) S += L - lens[c] + 1;
    const double d0 = gt_d0(L);
    const float k_tm = (float)(1.0 / (d0 * d0)), k_ms = 1.f / 12.25f;
    const float cut[5] = {1.f, 4.f, 12.25f, 16.f, 64.f};

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
            for (int i = s0; i < s0 + len; ++i) gt_add(mom, fa[i], fb[i]);
        int prev = -1, same = 0;
        for (int it = 0; it <= GT_MAX_REFINE && __any_sync(0xffffffffu, active); ++it) {
            float R32[9], tc[3], marg[5];
            if (active) {
                double R[9], t[3];
                gt_fit(mom, R, t);
#pragma unroll
                for (int k = 0; k < 9; ++k) s_rt[warp][k][lane] = R[k];
#pragma unroll
                for (int k = 0; k < 3; ++k) s_rt[warp][9 + k][lane] = t[k];
                // the fast path's frame: x = R cb + tc - ca with tc = R c_b + t - c_a
                float tmax = 0.f;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) R32[3 * r + c] = (float)R[3 * r + c];
                    tc[r] = (float)(R[3 * r] * cbx + R[3 * r + 1] * cby + R[3 * r + 2] * cbz + t[r] -
                                    (double)(r == 0 ? cax : (r == 1 ? cay : caz)));
                    tmax = fmaxf(tmax, fabsf(tc[r]));
                }
                // error bound of a component of x in FP32 (the rounded R and tc, the centring, the
                // fused steps: about 2^-24 (15 mc + 5 |tc|), taken 4x), then of d^2 near each cutoff
                // (2 sqrt(3) |x| dx + 3 dx^2 + the rounding of the sum of squares)
                const float dx = 32.f * 5.9604645e-8f * (2.f * mc + tmax);
#pragma unroll
                for (int k = 0; k < 5; ++k) marg[k] = 3.5f * sqrtf(cut[k]) * dx + 3.f * dx * dx + 4.8e-7f * cut[k];
            }
            GtMoments next;
            gt_zero(next);
            int c[4] = {0, 0, 0, 0};
            float tm = 0.f, ms = 0.f;
            if (active) {
                for (int i = 0; i < L; ++i) {
                    const float4 pa = ca[i], pb = cb[i];
                    const float x0 = fmaf(R32[0], pb.x, fmaf(R32[1], pb.y, fmaf(R32[2], pb.z, tc[0]))) - pa.x;
                    const float x1 = fmaf(R32[3], pb.x, fmaf(R32[4], pb.y, fmaf(R32[5], pb.z, tc[1]))) - pa.y;
                    const float x2 = fmaf(R32[6], pb.x, fmaf(R32[7], pb.y, fmaf(R32[8], pb.z, tc[2]))) - pa.z;
                    float d2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
                    bool near = false;
#pragma unroll
                    for (int k = 0; k < 5; ++k) near = near || fabsf(d2 - cut[k]) < marg[k];
                    bool in1 = d2 < 1.f, in2 = d2 < 4.f, in4 = d2 < 16.f, in8 = d2 < 64.f, sel = d2 < 12.25f;
                    if (near) {  // rare: the decision in FP64 from the given coordinates
                        const float4 ga = fa[i], gb = fb[i];
                        const double bv[3] = {gb.x, gb.y, gb.z}, av[3] = {ga.x, ga.y, ga.z};
                        double e2 = 0.0;
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            const double e = fma(s_rt[warp][3 * r][lane], bv[0],
                                                 fma(s_rt[warp][3 * r + 1][lane], bv[1],
                                                     fma(s_rt[warp][3 * r + 2][lane], bv[2], s_rt[warp][9 + r][lane]))) -
                                             av[r];
                            e2 = fma(e, e, e2);
                        }
                        in1 = e2 < 1.0;
                        in2 = e2 < 4.0;
                        in4 = e2 < 16.0;
                        in8 = e2 < 64.0;
                        sel = e2 < 12.25;
                        d2 = (float)e2;
                    }
                    c[0] += in1;
                    c[1] += in2;
                    c[2] += in4;
                    c[3] += in8;
                    // both terms from one approximate reciprocal, 1/qa = qb/(qa qb) and 1/qb = qa/(qa qb)
                    // (a few ulp each, far inside the FP32 sum's own rounding)
                    const float qa = fmaf(d2, k_tm, 1.f), qb = fmaf(d2, k_ms, 1.f);
                    const float rq = __fdividef(1.f, qa * qb);
                    tm = fmaf(qb, rq, tm);
                    ms = fmaf(qa, rq, ms);
                    if (sel) gt_add(next, fa[i], fb[i]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) best_c[k] = max(best_c[k], c[k]);
                best_tm = fmaxf(best_tm, tm);
                best_ms = fmaxf(best_ms, ms);
                const int ns = next.n;
                same = (ns == prev) ? same + 1 : 0;
                if (it == GT_MAX_REFINE || ns < 3 || same >= GT_STABLE || gt_equal(next, mom)) {
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
    const size_t smem = (size_t)L * 4 * sizeof(float4);
    cudaError_t e = cudaSuccess;
    // the static shared arrays (12.5 KB) count against the default 48 KB too, so the dynamic limit
    // is raised whenever the staged coordinates come near it
    if (smem > 32 * 1024) e = cudaFuncSetAttribute(gdt_tm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

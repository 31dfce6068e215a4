// bwd_tc.cuh -- pieces shared by the tensor-core adjoints (bwd_rot.cuh, bwd_rc.cuh):
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// The sweeps write one partial gradient slice per column range of B tiles (so that no CTA needs
// atomics on another's rows) and one partial row sum of w~ per slice; bwd_reduce_kernel adds the
// slices, the diagonal term (sum_b w~_ab) a and the centring projection. Here: the workspace of
// the stored-rotation adjoint (BtWs, carve_bt) and that reduction.
#pragma once
#include "backward.cuh"
#include "pairs_tc.cuh"
#include "rotation.cuh"

namespace clusco {

struct BtWs {
    float *xf = nullptr;     // [Rpad][Lp] centred FP32, padded row layout
    float *xT = nullptr;     // [2][Lp][Rpad] FP16 hi / lo parts, transposed (2 bytes each)
    float *Gp = nullptr;     // [S][Rpad][Lp] partial gradients
    float *dp = nullptr;     // [S][Npad] partial row sums of w~
    long long *nd_list = nullptr;
    unsigned long long *nd_count = nullptr;
    unsigned *scl = nullptr;  // max |centred x|, max |w| (float bits)
    int64_t S = 1, nd_cap = 0, Lp = 0, Npad = 0, Rpad = 0;
    size_t bytes = 0;
};

// Column ranges per A tile: enough CTAs for about four waves of 148 SMs.
inline int64_t bt_splits(int64_t TA, int64_t TB)
{
    int64_t S = (4 * 148 + TA - 1) / TA;
    if (S > TB) S = TB;
    return S < 1 ? 1 : S;
}

inline BtWs carve_bt(void *base, int64_t N, int64_t L)
{
    BtWs w;
    size_t off = 0;
    char *b = (char *)base;
    auto take = [&](size_t n) {
        void *p = b ? b + off : nullptr;
        off = (off + n + 255) & ~size_t(255);
        return p;
    };
    w.Lp = (L + 63) / 64 * 64;
    w.Npad = (N + TC_MA - 1) / TC_MA * TC_MA;
    w.Rpad = w.Npad / 10 * 32;
    w.S = bt_splits(w.Npad / TC_MA, w.Npad / TC_MB);
    w.xf = (float *)take(sizeof(float) * w.Rpad * w.Lp);
    w.xT = (float *)take((size_t)2 * 2 * w.Lp * w.Rpad);  // FP16 parts
    w.Gp = (float *)take(sizeof(float) * w.S * w.Rpad * w.Lp);
    w.dp = (float *)take(sizeof(float) * w.S * w.Npad);
    const int64_t P = N * (N - 1) / 2;
    w.nd_cap = nd_cap_for(P);
    w.nd_list = (long long *)take(sizeof(long long) * 2 * w.nd_cap);
    w.nd_count = (unsigned long long *)take(sizeof(unsigned long long));
    w.scl = (unsigned *)take(2 * sizeof(unsigned));
    w.bytes = off;
    return w;
}

// g_a = sum_s Gp[s] + (sum_s dp[s][a]) x_a, minus its atom mean. One block of three warps per
// model, warp = axis: each lane holds up to MAXQ float4 columns of its row (Lp <= 128 MAXQ),
// every partial slice is an independent 16-byte load, the axis mean is a warp reduction, and the
// model's gradient goes out through shared memory as one contiguous [L][3] run. Columns past L
// are zero in every input, so the row sum over Lp is the sum over L. S partial gradient slices,
// Sd partial row-sum slices.
constexpr int BRED_THREADS = 96;
constexpr int BRED_MAXQ = 4;

template <int MAXQ>
__global__ void __launch_bounds__(BRED_THREADS) bwd_reduce_kernel(const float *__restrict__ Gp,
                                                                  const float *__restrict__ dp,
                                                                  const float *__restrict__ xf, int64_t N, int L,
                                                                  int Lp, int64_t Rpad, int64_t S, int64_t Sd,
                                                                  float *__restrict__ grad)
{
    extern __shared__ float sg[];  // [L][3], as in grad
    const int lane = threadIdx.x & 31, ax = threadIdx.x >> 5;
    const int64_t a = blockIdx.x;
    const int64_t Npad = Rpad / 32 * 10;
    const int64_t row = tc_row(a, ax);
    const int64_t qslice = Rpad * (int64_t)Lp / 4;
    const float4 *g0 = reinterpret_cast<const float4 *>(Gp + row * Lp);
    const float4 *x0 = reinterpret_cast<const float4 *>(xf + row * Lp);
    const int nq = Lp / 4;
    float d = 0.f;
    for (int64_t s = 0; s < Sd; ++s) d += dp[s * Npad + a];
    float4 v[MAXQ];
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < MAXQ; ++c) {
        const int q = lane + 32 * c;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < nq) {
            const float4 x = __ldg(x0 + q);
            t = make_float4(d * x.x, d * x.y, d * x.z, d * x.w);
#pragma unroll 4
            for (int64_t s = 0; s < S; ++s) {
                const float4 gv = __ldg(g0 + s * qslice + q);
                t.x += gv.x;
                t.y += gv.y;
                t.z += gv.z;
                t.w += gv.w;
            }
        }
        v[c] = t;
        m += (t.x + t.y) + (t.z + t.w);
    }
    m = warp_sum_f(m) / (float)L;
#pragma unroll
    for (int c = 0; c < MAXQ; ++c) {
        const int i = 4 * (lane + 32 * c);
        if (i + 0 < L) sg[3 * (i + 0) + ax] = v[c].x - m;
        if (i + 1 < L) sg[3 * (i + 1) + ax] = v[c].y - m;
        if (i + 2 < L) sg[3 * (i + 2) + ax] = v[c].z - m;
        if (i + 3 < L) sg[3 * (i + 3) + ax] = v[c].w - m;
    }
    __syncthreads();
    float *ga = grad + a * (int64_t)L * 3;
    for (int e = threadIdx.x; e < 3 * L; e += BRED_THREADS) ga[e] = sg[e];
}

inline cudaError_t launch_bwd_reduce(const BtWs &w, int64_t N, int64_t L, float *grad, cudaStream_t st)
{
    bwd_reduce_kernel<BRED_MAXQ><<<(unsigned)N, BRED_THREADS, (size_t)(3 * L * sizeof(float)), st>>>(
        w.Gp, w.dp, w.xf, N, (int)L, (int)w.Lp, w.Rpad, w.S, w.S, grad);
    return cudaGetLastError();
}

}  // namespace clusco

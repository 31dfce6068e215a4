// bwd_tc.cuh -- adjoint of the all-pairs matrix with the covariance recomputed on tcgen05.
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// One CTA (8 warps, 255 registers each) owns one A tile I (40 models = 128 rows of the operand planes) and a
// contiguous range of B tiles J over the full square (every b != a, both orders, so each
// CTA owns its rows and needs no atomics). For every J:
//   1. the exact-digit covariance of the 40 x 20 tile is recomputed on the tensor cores
//      (TMA -> 2-stage ring -> tcgen05.mma -> TMEM, as in the forward kernel);
//   2. the warps read TMEM, build each 3x3 block (rows cyclic, as in the forward), take
//      Sigma from the FP32 fast path and the optimal rotation from Horn's quaternion form,
//      undo the cyclic row order, and write w~ R into the shared tile P^T (64 x 128); pairs
//      below the near-duplicate threshold are queued for the FP64 direct kernel instead;
//      meanwhile one bulk TMA copy brings the FP32 centred coordinates of the 20 B models
//      (64 contiguous rows of the FP32 plane) into shared memory;
//   3. the warps contract: G_I(128 rows x Lp atoms) -= P (128 x 64) . X_J (64 x Lp), in
//      FP32, with G_I held in registers (16 rows x Lp/32 atoms per thread) for the whole
//      sweep over J. Rotations are never written to global memory.
// The CTA finally stores its partial G_I and its row sums of w~; bwd_reduce_kernel adds
// the partials of the S column ranges, the diagonal term and the centring projection.
// L is limited to 320 atoms (Lp <= 320) by the register-resident accumulators.
#pragma once
#include "backward.cuh"
#include "pairs_tc.cuh"
#include "rotation.cuh"

namespace clusco {

constexpr int BT_THREADS = 256;
constexpr int BT_ROWS = 128 / (BT_THREADS / 32);  // accumulator rows per thread
constexpr int BT_MAXLP = 320;
constexpr size_t BT_RING = TC_STAGES * STAGE_BYTES_BF16;
constexpr size_t BT_XS = (size_t)64 * BT_MAXLP * 4;
constexpr size_t BT_PS = (size_t)64 * 128 * 4;
constexpr size_t BT_SMEM = 1024 + BT_RING + BT_XS + BT_PS;

struct BtWs {
    void *planes = nullptr;  // EXACT2 digit planes [2][Rpad][Lp] bf16
    float *scales = nullptr;
    double *G64 = nullptr;
    float *G32 = nullptr;
    float *xf = nullptr;   // [Rpad][Lp] centred FP32, padded row layout
    float *Gp = nullptr;   // [S][Rpad][Lp] partial gradients
    float *dp = nullptr;   // [S][Npad] partial row sums of w~
    long long *nd_list = nullptr;
    unsigned long long *nd_count = nullptr;
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
    w.planes = take((size_t)2 * w.Rpad * w.Lp * 2);
    w.scales = (float *)take(sizeof(float) * 3 * w.Npad);
    w.G64 = (double *)take(sizeof(double) * w.Npad);
    w.G32 = (float *)take(sizeof(float) * w.Npad);
    w.xf = (float *)take(sizeof(float) * w.Rpad * w.Lp);
    w.Gp = (float *)take(sizeof(float) * w.S * w.Rpad * w.Lp);
    w.dp = (float *)take(sizeof(float) * w.S * w.Npad);
    const int64_t P = N * (N - 1) / 2;
    w.nd_cap = P < (int64_t)(1 << 22) ? P : (int64_t)(1 << 22);
    w.nd_list = (long long *)take(sizeof(long long) * 2 * w.nd_cap);
    w.nd_count = (unsigned long long *)take(sizeof(unsigned long long));
    w.bytes = off;
    return w;
}

template <int NJ>
__global__ void __launch_bounds__(BT_THREADS, 1)
    bwd_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const float *__restrict__ scales, const float *__restrict__ G32, const float *__restrict__ xf,
                  int64_t N, int L, int Lp, int nkb, int64_t Rpad, int64_t TB, int64_t S, int64_t JC,
                  const float *__restrict__ crmsd, const float *__restrict__ wvec, float eps,
                  float *__restrict__ Gp, float *__restrict__ dp, long long *__restrict__ nd_list,
                  unsigned long long *__restrict__ nd_count, int64_t nd_cap)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ __align__(8) uint64_t xs_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float sB_scale[TC_MB * 3];
    __shared__ float sB_G32[TC_MB];
    __shared__ float dsum[TC_MA];

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase0 = smem_u32(smem);
    float *Xs = reinterpret_cast<float *>(smem + BT_RING);          // [64][Lp]
    float *PsT = reinterpret_cast<float *>(smem + BT_RING + BT_XS);  // [64][128]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t I = blockIdx.x / S, sidx = blockIdx.x % S;
    const int64_t J0 = sidx * JC, J1 = (J0 + JC < TB) ? J0 + JC : TB;
    const int64_t a_base = I * TC_MA;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, TC_TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        mbar_init(&xs_bar, 1);
        abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    for (int e = tid; e < 64 * 128; e += BT_THREADS) PsT[e] = 0.f;
    if (tid < TC_MA) dsum[tid] = 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // epilogue-side constants (warps 0-7)
    const int sp = warp & 3, g = (warp >> 2) & 1;
    const int mloc = lane / 3, alpha = lane - 3 * (lane / 3);
    const int la = 10 * sp + mloc;
    const int64_t a = a_base + la;
    const bool lane_ok = lane < 30 && a < N;
    float srow0 = 1.f, Ga = 0.f;
    if (lane_ok) {
        srow0 = scales[a * 3 + alpha];
        Ga = G32[a];
    }
    const uint32_t trow = tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)(32 * g);
    const float invL = 1.f / (float)L;

    // contraction-side: rows BT_ROWS*rg .. +BT_ROWS-1 of the tile, atoms lane + 32 j
    const int rg = warp;
    float acc[BT_ROWS][NJ];
#pragma unroll
    for (int r = 0; r < BT_ROWS; ++r)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[r][j] = 0.f;

    int64_t kbt = 0;
    bool alive = true;
    for (int64_t J = J0; J < J1 && alive; ++J) {
        const int64_t jt = J - J0;
        const int64_t b_base = J * TC_MB;
        if (tid < TC_MB * 3) sB_scale[tid] = scales[(b_base + tid / 3) * 3 + tid % 3];
        if (tid < TC_MB) sB_G32[tid] = G32[b_base + tid];
        // ---- 1. covariance of the tile on the tensor cores ----
        if (warp == 0 && lane == 0) {
            // the B tile's FP32 coordinates: 64 contiguous rows of the FP32 plane
            mbar_arrive_expect_tx(&xs_bar, (uint32_t)(64 * Lp * 4));
            bulk_load(Xs, xf + (64 * J) * (int64_t)Lp, (uint32_t)(64 * Lp * 4), &xs_bar);
            for (int kb = 0; kb < nkb; ++kb) {
                const int64_t q = kbt + kb;
                const int s = (int)(q % TC_STAGES);
                const int64_t use = q / TC_STAGES;
                if (q >= TC_STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                uint8_t *st = smem + s * STAGE_BYTES_BF16;
                mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES_BF16);
                const int x = kb * 64;
                tma_load_2d(st, &mapA, &full_bar[s], x, (int)(128 * I));
                tma_load_2d(st + 16384, &mapA, &full_bar[s], x, (int)(Rpad + 128 * I));
                tma_load_2d(st + 32768, &mapB, &full_bar[s], x, (int)(64 * J));
                tma_load_2d(st + 40960, &mapB, &full_bar[s], x, (int)(Rpad + 64 * J));
            }
        } else if (warp == 1 && lane == 0) {
            for (int kb = 0; kb < nkb; ++kb) {
                const int64_t q = kbt + kb;
                const int s = (int)(q % TC_STAGES);
                const int64_t use = q / TC_STAGES;
                if (!mbar_wait(&full_bar[s], (uint32_t)(use & 1)) || *(volatile int *)&abort_flag) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                tc_fence_after();
                tc_issue_kblock<TC_EXACT2>(tmem, sbase0 + s * STAGE_BYTES_BF16, kb);
                mma_commit(&empty_bar[s]);
            }
            mma_commit(&done_bar);
        }
        kbt += nkb;
        __syncwarp();
        if (!mbar_wait_sleep(&done_bar, (uint32_t)(jt & 1))) atomicExch(&abort_flag, 1);
        tc_fence_after();
        __syncthreads();
        if (*(volatile int *)&abort_flag) {  // read after the barrier: a uniform decision
            alive = false;
            break;
        }
        {
            // ---- 2. rotations of the tile's pairs into P^T ----
            float V[32];
            {
                float t[32];
                tmem_ld32(trow + 0, V);
#pragma unroll
                for (int j = 0; j < 32; ++j) V[j] *= 65536.f;
                tmem_ld32(trow + 64, t);
#pragma unroll
                for (int j = 0; j < 32; ++j) V[j] = fmaf(256.f, t[j], V[j]);
                tmem_ld32(trow + 128, t);
#pragma unroll
                for (int j = 0; j < 32; ++j) V[j] = fmaf(256.f, t[j], V[j]);
                tmem_ld32(trow + 192, t);
#pragma unroll
                for (int j = 0; j < 32; ++j) V[j] += t[j];
#pragma unroll
                for (int j = 0; j < 30; ++j) V[j] *= srow0 * sB_scale[30 * g + j];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float cand[3][3];
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) {
                        const int j = 9 * r + 3 * al + be;
                        cand[al][be] = (j < 32) ? V[j] : 0.f;
                    }
                float blk[9];
#pragma unroll
                for (int be = 0; be < 3; ++be) blk[be] = sel3(alpha, cand[0][be], cand[1][be], cand[2][be]);
#pragma unroll
                for (int k = 1; k <= 2; ++k) {
                    const int sendsel = (alpha + 3 - k) % 3;
                    const int src = 3 * mloc + (alpha + k) % 3;
#pragma unroll
                    for (int be = 0; be < 3; ++be)
                        blk[3 * k + be] = __shfl_sync(0xffffffffu, sel3(sendsel, cand[0][be], cand[1][be], cand[2][be]),
                                                      src & 31);
                }
                const int bq = 3 * r + alpha;  // local B model within the group
                if (lane < 30 && bq < 10) {
                    const int lb = 10 * g + bq;
                    const int64_t b = b_base + lb;
                    float P[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                    if (lane_ok && b < N && b != a) {
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
                            float sfast, errc2;
                            const float Gb = sB_G32[lb];
                            crmsd_fast_fp32(blk, Ga, Gb, invL, &sfast, &errc2);
                            const float nrm = __fdividef(2.f, Ga + Gb);
                            float Hn[9], Rp[9];
#pragma unroll
                            for (int e = 0; e < 9; ++e) Hn[e] = blk[e] * nrm;
                            horn_rotation(Hn, sfast, Rp);
                            const float coef = w / ((float)L * fmaxf(c, eps));
                            // undo the cyclic row order: row i of R is row (i - alpha) mod 3 of Rp
#pragma unroll
                            for (int i = 0; i < 3; ++i) {
                                const int src_row = (i + 3 - alpha) % 3;
#pragma unroll
                                for (int be = 0; be < 3; ++be)
                                    P[3 * i + be] = coef * sel3(src_row, Rp[be], Rp[3 + be], Rp[6 + be]);
                            }
                            atomicAdd(&dsum[la], coef);
                        }
                    }
                    // P^T[col(b, beta)][row(a, i)]
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int be = 0; be < 3; ++be)
                            PsT[(32 * g + 3 * bq + be) * 128 + 32 * sp + 3 * mloc + i] = P[3 * i + be];
                }
            }
        }
        if (!mbar_wait_sleep(&xs_bar, (uint32_t)(jt & 1))) atomicExch(&abort_flag, 1);
        tc_fence_before();
        __syncthreads();
        if (*(volatile int *)&abort_flag) {
            alive = false;
            break;
        }
        // ---- 3. contraction G_I -= P . X_J over the 60 real rows of the B tile ----
#pragma unroll 1
        for (int gq = 0; gq < 2; ++gq) {
#pragma unroll 2
            for (int q = 0; q < 30; ++q) {
                const int k = 32 * gq + q;
                float pv[BT_ROWS];
#pragma unroll
                for (int r4 = 0; r4 < BT_ROWS / 4; ++r4) {
                    const float4 p = *reinterpret_cast<const float4 *>(PsT + k * 128 + BT_ROWS * rg + 4 * r4);
                    pv[4 * r4] = p.x;
                    pv[4 * r4 + 1] = p.y;
                    pv[4 * r4 + 2] = p.z;
                    pv[4 * r4 + 3] = p.w;
                }
                float xv[NJ];
#pragma unroll
                for (int j = 0; j < NJ; ++j) xv[j] = Xs[k * Lp + lane + 32 * j];
#pragma unroll
                for (int r = 0; r < BT_ROWS; ++r)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) acc[r][j] = fmaf(-pv[r], xv[j], acc[r][j]);
            }
        }
        __syncthreads();
    }
    if (!alive) {
        // drain: wait (bounded) for the loads this CTA issued before giving up
        if (warp == 0 && lane == 0 && kbt > 0) {
            for (int64_t q = (kbt > TC_STAGES ? kbt - TC_STAGES : 0); q < kbt; ++q)
                mbar_wait(&full_bar[q % TC_STAGES], (uint32_t)((q / TC_STAGES) & 1));
            mbar_wait(&xs_bar, (uint32_t)(((kbt / nkb) - 1) & 1));
        }
    } else {
        float *gp = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
#pragma unroll
        for (int r = 0; r < BT_ROWS; ++r)
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int atom = lane + 32 * j;
                if (atom < Lp) gp[(BT_ROWS * rg + r) * (int64_t)Lp + atom] = acc[r][j];
            }
        if (tid < TC_MA) dp[sidx * (Rpad / 32 * 10) + a_base + tid] = dsum[tid];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

// g_a = sum_s Gp[s] + (sum_s dp[s][a]) x_a, minus its atom mean; one warp per model.
__global__ void __launch_bounds__(256) bwd_reduce_kernel(const float *__restrict__ Gp, const float *__restrict__ dp,
                                                         const float *__restrict__ xf, int64_t N, int L, int Lp,
                                                         int64_t Rpad, int64_t S, float *__restrict__ grad)
{
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (a >= N) return;
    const int64_t Npad = Rpad / 32 * 10;
    float d = 0.f;
    for (int64_t s = 0; s < S; ++s) d += dp[s * Npad + a];
    for (int ax = 0; ax < 3; ++ax) {
        const int64_t row = tc_row(a, ax);
        float m = 0.f;
        for (int i = lane; i < L; i += 32) {
            float v = d * xf[row * Lp + i];
            for (int64_t s = 0; s < S; ++s) v += Gp[(s * Rpad + row) * Lp + i];
            m += v;
        }
        m = warp_sum_f(m) / (float)L;
        for (int i = lane; i < L; i += 32) {
            float v = d * xf[row * Lp + i];
            for (int64_t s = 0; s < S; ++s) v += Gp[(s * Rpad + row) * Lp + i];
            grad[(a * L + i) * 3 + ax] = v - m;
        }
    }
}

}  // namespace clusco

namespace clusco {

// Host side: pre-pass (digits + FP32 copy), the tensor-core sweep, the reduction, and the
// FP64 near-duplicate kernel. Requires L <= 320 and an sm_103 device.
inline int bt_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                     float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
{
    const BtWs w = carve_bt(ws, N, L);
    const unsigned pblocks = (unsigned)((w.Npad + 7) / 8);
    prepass_tc_kernel<TC_EXACT2><<<pblocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Rpad, w.planes,
                                                           w.scales, w.G64, w.G32, w.xf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(w.nd_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
        err = std::string("backward pre-pass: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    CUtensorMap mA, mB;
    int rc;
    if ((rc = make_map(&mA, w.planes, false, w.Lp, 2 * w.Rpad, 128, err))) return rc;
    if ((rc = make_map(&mB, w.planes, false, w.Lp, 2 * w.Rpad, 64, err))) return rc;
    const int64_t TA = w.Npad / TC_MA, TB = w.Npad / TC_MB;
    const int64_t JC = (TB + w.S - 1) / w.S;
    const int nkb = (int)(w.Lp / 64);
    const unsigned grid = (unsigned)(TA * w.S);
#define CLUSCO_BT_CASE(NJ_)                                                                                      \
    case NJ_:                                                                                                    \
        e = cudaFuncSetAttribute(bwd_tc_kernel<NJ_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BT_SMEM);  \
        if (e == cudaSuccess)                                                                                    \
            bwd_tc_kernel<NJ_><<<grid, BT_THREADS, BT_SMEM, st>>>(mA, mB, w.scales, w.G32, w.xf, N, (int)L,       \
                                                                  (int)w.Lp, nkb, w.Rpad, TB, w.S, JC, crmsd,      \
                                                                  grad_out, eps, w.Gp, w.dp, w.nd_list, w.nd_count, \
                                                                  w.nd_cap);                                       \
        break;
    switch ((int)(w.Lp / 32)) {
        CLUSCO_BT_CASE(2)
        CLUSCO_BT_CASE(4)
        CLUSCO_BT_CASE(6)
        CLUSCO_BT_CASE(8)
        CLUSCO_BT_CASE(10)
    default:
        err = "tensor-core backward needs L <= 320";
        return CLUSCO_EUNSUPPORTED;
    }
#undef CLUSCO_BT_CASE
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        bwd_reduce_kernel<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(w.Gp, w.dp, w.xf, N, (int)L, (int)w.Lp, w.Rpad,
                                                                    w.S, grad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bwd_neardup_kernel<<<296, 256, 0, st>>>(coords, N, (int)L, grad_out, eps, w.nd_list, w.nd_count, w.nd_cap,
                                                grad);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("tensor-core backward: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

}  // namespace clusco

namespace clusco {

inline size_t backward_ws_bytes(int64_t N, int64_t L, int form)
{
    (void)form;
    size_t a = backward_simt_ws_bytes(N, L);
    if (L <= BT_MAXLP) {
        const size_t b = carve_bt(nullptr, N, L).bytes;
        if (b > a) a = b;
    }
    return a;
}

// The adjoint: tensor-core recompute when the device and L allow it, else the CUDA-core path.
inline int backward_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                           float *grad, float eps, int form, void *ws, cudaStream_t st, std::string &err)
{
    if (L <= BT_MAXLP && tc_supported(CLUSCO_FORM_BF16_EXACT2, L) == CLUSCO_OK)
        return bt_launch(coords, N, L, grad_out, crmsd, grad, eps, ws, st, err);
    return backward_simt_launch(coords, N, L, grad_out, crmsd, grad, eps, form, ws, st, err);
}

}  // namespace clusco

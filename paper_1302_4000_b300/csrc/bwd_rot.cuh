// bwd_rot.cuh -- adjoint of the all-pairs matrix from stored rotations (tcgen05 contraction only).
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// The forward can store each pair's optimal rotation R_ab (pairs_tc_kernel with ROT); then the
// adjoint needs no covariance and no rotation arithmetic: per tile it only gathers R_ab (or
// R_ba^T for the lower triangle), c_ab and w_ab, scales, and contracts. Same tiling as
// bwd_tc_kernel: a CTA owns one A tile I (40 models = 128 operand rows) and a contiguous range
// of B tiles J over the full square (every b != a in both orders, so no atomics on the
// gradient). Roles:
//   warp 0 (TMA): X_J^T hi / lo TF32 chunks (128 atoms x 32 operand rows) into a 3-stage ring;
//   warp 1 (MMA): the contraction transposed, sum^T += X_J^T . P_J^T (tcgen05 kind::tf32,
//     M = 128 atoms, N = 128 rows of the A tile, three passes hi.hi + hi.lo + lo.hi): with the
//     atoms as M the MMAs are 128 x 128 instead of 128 x 64, and the same shared P operand
//     serves as the K-major B operand. The accumulator holds ceil(Lp/128) blocks of 128
//     columns (TMEM lanes = atoms);
//   warps 2-9 (epilogue): each lane owns one row (model a, axis alpha) of the tile's 128 x 64
//     operand: it gathers row alpha of R_ab (or column alpha of R_ba) and c, w for its ten
//     B models, scales, and stores the row as two TF32 parts with 16-byte stores into one of
//     two shared operands (128-byte swizzle, K-major), so that tile J+1's operand is written
//     while GEMM2 reads tile J's. Pairs below the near-duplicate threshold go to the FP64
//     direct kernel, as in the recompute path.
// At the end the CTA's sum goes out of TMEM into its partial slice; bwd_reduce_kernel adds the
// partials, the diagonal term and the centring projection.
#pragma once
#include "bwd_tc.cuh"

namespace clusco {

constexpr int BR_THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int BR_XSTAGES = 3;
constexpr int BR_MAXLP = 512;
constexpr int BR_ABLK = 128;                      // atoms per accumulator block (MMA M)
constexpr size_t BR_XBUF = 2 * 32 * BR_ABLK * 4;  // hi, lo: 32 operand rows x 128 atoms, 32 KB
constexpr size_t BR_SMEM = 1024 + 2 * BT_A2 + BR_XSTAGES * BR_XBUF;  // 1 KB + 128 KB + 96 KB
static_assert(BR_SMEM <= 227 * 1024, "shared memory per CTA");

__global__ void __launch_bounds__(BR_THREADS, 1)
    bwd_rot_kernel(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl, int64_t N,
                   int L, int Lp, uint32_t tmem_cols,
                   int64_t Rpad, int64_t TB, int64_t S, int64_t JC, const float *__restrict__ crmsd,
                   const float *__restrict__ wvec, const float *__restrict__ rot, float eps, float *__restrict__ Gp,
                   float *__restrict__ dp, long long *__restrict__ nd_list, unsigned long long *__restrict__ nd_count,
                   int64_t nd_cap)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t xfull_bar[BR_XSTAGES];   // an X^T chunk landed
    __shared__ __align__(8) uint64_t xempty_bar[BR_XSTAGES];  // GEMM2 has finished reading it
    __shared__ __align__(8) uint64_t a2full_bar[2];           // a rotation operand is written (8 arrivals)
    __shared__ __align__(8) uint64_t a2empty_bar[2];          // GEMM2 has finished reading it
    __shared__ __align__(8) uint64_t d2_bar;                  // the last GEMM2 has finished
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float dsum[TC_MA];

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *A2 = smem;                // two operands of BT_A2 bytes: [hi 32 KB][lo 32 KB] each
    uint8_t *XT = smem + 2 * BT_A2;    // BR_XSTAGES chunk buffers of BT_XBUF bytes
    const uint32_t a2base = smem_u32(A2), xtbase = smem_u32(XT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t I = blockIdx.x / S, sidx = blockIdx.x % S;
    const int64_t J0 = sidx * JC, J1 = (J0 + JC < TB) ? J0 + JC : TB;
    const int64_t a_base = I * TC_MA;
    const int64_t Npad = Rpad / 32 * 10;

    if (J0 >= J1) {  // an empty column range still owns its (zero) partial slice
        float *gp = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
        for (int e = tid; e < 128 * Lp; e += BR_THREADS) gp[e] = 0.f;
        if (tid < TC_MA) dp[sidx * Npad + a_base + tid] = 0.f;
        return;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, tmem_cols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < BR_XSTAGES; ++s) {
            mbar_init(&xfull_bar[s], 1);
            mbar_init(&xempty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a2full_bar[b], 8);
            mbar_init(&a2empty_bar[b], 1);
        }
        mbar_init(&d2_bar, 1);
        abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    // pad rows and columns of both operands stay zero for the whole sweep
    for (int e = tid; e < (int)(2 * BT_A2 / 16); e += BR_THREADS)
        reinterpret_cast<float4 *>(A2)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < TC_MA) dsum[tid] = 0.f;
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int64_t nJ = J1 - J0;
    const int nblk = (Lp + BR_ABLK - 1) / BR_ABLK;
    const int nch = 2 * nblk;  // per tile: atom blocks x the two 32-row halves of the B tile
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        // ================= TMA producer: X^T chunks =================
        if (lane == 0) {
            int64_t c = 0;
            bool ok = true;
            for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) {
                const int64_t J = J0 + j;
                for (int ch = 0; ch < nch && ok; ++ch, ++c) {
                    const int st = (int)(c % BR_XSTAGES);
                    const int64_t use = c / BR_XSTAGES;
                    if (c >= BR_XSTAGES && !mbar_wait_sleep(&xempty_bar[st], (uint32_t)((use - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    // chunk ch = (atom block ch / 2, operand-row half ch % 2); atoms past Lp read zeros
                    const int x = (int)(64 * J + 32 * (ch & 1)), y = (ch >> 1) * BR_ABLK;
                    mbar_arrive_expect_tx(&xfull_bar[st], (uint32_t)BR_XBUF);
                    tma_load_2d(XT + st * BR_XBUF, &mapXh, &xfull_bar[st], x, y);
                    tma_load_2d(XT + st * BR_XBUF + BR_XBUF / 2, &mapXl, &xfull_bar[st], x, y);
                }
            }
            if (!ok) atomicExch(&abort_flag, 1);
            if (*abort_v) {
                // loads still in flight must land before the CTA leaves (bounded waits)
                for (int64_t r = (c > BR_XSTAGES ? c - BR_XSTAGES : 0); r < c; ++r)
                    mbar_wait(&xfull_bar[r % BR_XSTAGES], (uint32_t)((r / BR_XSTAGES) & 1));
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ================= MMA issuer: GEMM2 only =================
        if (lane == 0) {
            int64_t c = 0;
            bool ok = true;
            constexpr uint32_t idx = make_idesc(BR_ABLK, 128, 2);
            for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) {
                const int buf = (int)(j & 1);
                if (!mbar_wait_sleep(&a2full_bar[buf], (uint32_t)((j >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ab = a2base + (uint32_t)(buf * BT_A2);
                for (int ch = 0; ch < nch && ok; ++ch, ++c) {
                    const int st = (int)(c % BR_XSTAGES);
                    if (!mbar_wait(&xfull_bar[st], (uint32_t)((c / BR_XSTAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xb = xtbase + st * BR_XBUF;
                    const int kh = ch & 1;
                    const uint32_t d = tmem + (uint32_t)((ch >> 1) * 128);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        // A = X^T (atoms x operand rows), B = P (A-tile rows x operand rows), both K-major
                        const uint64_t xhi = desc_sw128(xb + 32 * k);
                        const uint64_t xlo = desc_sw128(xb + BR_XBUF / 2 + 32 * k);
                        const uint64_t phi = desc_sw128(ab + kh * 16384 + 32 * k);
                        const uint64_t plo = desc_sw128(ab + 32768 + kh * 16384 + 32 * k);
                        // each block's first MMA of the sweep starts its columns from zero
                        mma_tf32(d, xhi, phi, idx, (j == 0 && kh == 0 && k == 0) ? 0u : 1u);
                        mma_tf32(d, xhi, plo, idx, 1u);
                        mma_tf32(d, xlo, phi, idx, 1u);
                    }
                    mma_commit(&xempty_bar[st]);
                }
                mma_commit(&a2empty_bar[buf]);
            }
            mma_commit(&d2_bar);  // also on abort: fires once everything issued has finished
            if (!mbar_wait(&d2_bar, 0)) ok = false;
            if (!ok) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else {
        // ================= epilogue warps 2..9 =================
        const int etid = tid - 64;
        const int sp = warp & 3, g = (warp - 2) >> 2;
        const int mloc = lane / 3, alpha = lane - 3 * (lane / 3);
        const int la = 10 * sp + mloc;
        const int64_t a = a_base + la;
        const bool lane_ok = lane < 30 && a < N;
        const float fL = (float)L;
        bool alive = true;
        // This lane owns row (a, alpha) of each tile's operand: for each of its half's 10 B
        // models b, row alpha of w~ R_ab (or column alpha of R_ba when a > b). The gathers (c, w
        // and three floats of each record) are software-pipelined: tile j+1's are issued before
        // tile j's operand is stored, so their latency overlaps the wait and the stores.
        float cg[10], wg[10], rg[10][3];
        auto gather = [&](int64_t jj) {
            const int64_t gb = (J0 + jj) * TC_MB + 10 * g;
#pragma unroll
            for (int bq = 0; bq < 10; ++bq) {
                const int64_t b = gb + bq;
                cg[bq] = 0.f;
                wg[bq] = 0.f;
                rg[bq][0] = rg[bq][1] = rg[bq][2] = 0.f;
                if (lane_ok && b < N && b != a) {
                    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
                    const int64_t idx = condensed_idx(lo, hi, N);
                    cg[bq] = __ldg(crmsd + idx);
                    wg[bq] = __ldg(wvec + idx);
                    const float *rec = rot + idx * ROT_STRIDE;
                    // R_ab row alpha = rec[3 alpha + be]; R_ba^T row alpha = rec[3 be + alpha]
                    const int o0 = a < b ? 3 * alpha : alpha, st = a < b ? 1 : 3;
                    rg[bq][0] = __ldg(rec + o0);
                    rg[bq][1] = __ldg(rec + o0 + st);
                    rg[bq][2] = __ldg(rec + o0 + 2 * st);
                }
            }
        };
        gather(0);
        for (int64_t j = 0; j < nJ; ++j) {
            const int64_t b_base = (J0 + j) * TC_MB;
            const int buf = (int)(j & 1);
            float v[32];
            float csum = 0.f;
#pragma unroll
            for (int bq = 0; bq < 10; ++bq) {
                const int64_t b = b_base + 10 * g + bq;
                float coef = 0.f;
                if (lane_ok && b < N && b != a) {
                    const float c = cg[bq], w = wg[bq];
                    if (!(c >= CLUSCO_NEARDUP)) {
                        if (alpha == 0 && a < b && w != 0.f) {  // one lane per pair queues it
                            const unsigned long long slot = atomicAdd(nd_count, 1ull);
                            if ((int64_t)slot < nd_cap) {
                                nd_list[2 * slot] = a;
                                nd_list[2 * slot + 1] = b;
                            }
                        }
                    } else if (w != 0.f) {
                        coef = __fdividef(w, fL * fmaxf(c, eps));
                    }
                }
                csum += coef;
#pragma unroll
                for (int be = 0; be < 3; ++be) v[3 * bq + be] = coef * rg[bq][be];
            }
            v[30] = v[31] = 0.f;
            if (alpha == 0 && lane_ok) atomicAdd(&dsum[la], csum);
            if (j + 1 < nJ) gather(j + 1);  // consumed by the next iteration
            // the operand buffer is reused every other tile: wait until GEMM2 of tile j-2 read it
            bool ok2 = true;
            if (j >= 2) ok2 = mbar_wait_sleep(&a2empty_bar[buf], (uint32_t)(((j >> 1) - 1) & 1));
            if (named_bar_or(1, 256, !ok2 || *abort_v)) {
                alive = false;
                break;
            }
            // the row, as two TF32 parts, into the 128-byte-swizzled K-major operand: row
            // 32 sp + lane of column block g, eight 16-byte chunks at (chunk ^ (row mod 8))
            if (lane < 30) {
                const int row = 32 * sp + lane;
                uint8_t *base = A2 + buf * BT_A2 + g * 16384 + row * 128;
#pragma unroll
                for (int c16 = 0; c16 < 8; ++c16) {
                    float h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        h[e] = tf32_rna(v[4 * c16 + e]);
                        l[e] = tf32_rna(v[4 * c16 + e] - h[e]);
                    }
                    const int off = ((c16 ^ (row & 7)) & 7) << 4;
                    *reinterpret_cast<float4 *>(base + off) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4 *>(base + 32768 + off) = make_float4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_proxy_async();  // generic-proxy stores to the operand must be visible to tcgen05.mma
            __syncwarp();
            if (lane == 0) mbar_arrive(&a2full_bar[buf]);
        }
        if (alive) {
            const bool ok3 = mbar_wait_sleep(&d2_bar, 0);
            if (named_bar_or(1, 256, !ok3 || *abort_v)) alive = false;
        }
        if (alive) {
            tc_fence_after();
            // read the transposed sum out of TMEM: warp (sp, g) takes TMEM lanes 32 sp.. (atoms)
            // and half g of each block's 128 columns (rows of the A tile)
            float *gbase = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
            for (int blk = 0; blk < nblk; ++blk) {
                const int atom = blk * BR_ABLK + 32 * sp + lane;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r0 = 64 * g + 32 * h;
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)(blk * 128 + r0), v);
                    if (atom < Lp) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) gbase[(int64_t)(r0 + jj) * Lp + atom] = -v[jj];
                    }
                }
            }
            if (etid < TC_MA) dp[sidx * Npad + a_base + etid] = dsum[etid];
        } else {
            atomicExch(&abort_flag, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

inline bool bwr_supported(int64_t L) { return (L + 63) / 64 * 64 <= BR_MAXLP; }

// Host side: pre-pass (FP32 copy + transposed TF32 parts), the contraction sweep from stored
// rotations, the reduction, and the FP64 near-duplicate kernel. Workspace: carve_bt's layout.
inline int bwr_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                      const float *rot, float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
{
    const BtWs w = carve_bt(ws, N, L);
    const unsigned pblocks = (unsigned)((w.Npad + 7) / 8);
    prepass_tc_kernel<TC_EXACT2><<<pblocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Rpad, w.planes,
                                                           w.scales, w.G64, w.G32, w.xf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        bt_transpose_kernel<<<dim3((unsigned)(w.Rpad / 32), (unsigned)(w.Lp / 32)), 256, 0, st>>>(w.xf, w.Rpad,
                                                                                                 (int)w.Lp, w.xT);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(w.nd_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
        err = std::string("backward pre-pass: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    CUtensorMap mXh, mXl;
    for (int part = 0; part < 2; ++part) {
        // X^T hi / lo parts: FP32 [Lp][Rpad] each; boxes of 32 operand rows (128 bytes) x 128
        // atoms; atoms past Lp read as zeros
        const cuuint64_t dims[2] = {(cuuint64_t)w.Rpad, (cuuint64_t)w.Lp};
        const cuuint64_t strides[1] = {(cuuint64_t)(w.Rpad * 4)};
        const cuuint32_t box[2] = {32u, (cuuint32_t)BR_ABLK};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(part ? &mXl : &mXh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, w.xT + part * w.Lp * w.Rpad,
                                 dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            err = "cuTensorMapEncodeTiled (X^T) failed (" + std::to_string((int)r) + ")";
            return CLUSCO_ECUDA;
        }
    }
    const int64_t TA = w.Npad / TC_MA, TB = w.Npad / TC_MB;
    const int64_t JC = (TB + w.S - 1) / w.S;
    uint32_t cols = 32;
    const uint32_t need_cols = (uint32_t)((w.Lp + BR_ABLK - 1) / BR_ABLK * 128);
    while (cols < need_cols) cols <<= 1;  // TMEM allocations are powers of two
    const unsigned grid = (unsigned)(TA * w.S);
    e = cudaFuncSetAttribute(bwd_rot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BR_SMEM);
    if (e == cudaSuccess) {
        prof_mark(PROF_ADJOINT, st);
        bwd_rot_kernel<<<grid, BR_THREADS, BR_SMEM, st>>>(mXh, mXl, N, (int)L, (int)w.Lp, cols, w.Rpad, TB, w.S, JC, crmsd,
                                                          grad_out, rot, eps, w.Gp, w.dp, w.nd_list, w.nd_count,
                                                          w.nd_cap);
        e = cudaGetLastError();
        prof_mark(PROF_ADJOINT, st);
    }
    if (e == cudaSuccess) {
        bwd_reduce_kernel<<<(unsigned)((3 * N + 7) / 8), 256, 0, st>>>(w.Gp, w.dp, w.xf, N, (int)L, (int)w.Lp, w.Rpad,
                                                                    w.S, grad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bwd_neardup_kernel<<<296, 256, 0, st>>>(coords, N, (int)L, grad_out, eps, w.nd_list, w.nd_count, w.nd_cap,
                                                grad);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("backward from stored rotations: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

}  // namespace clusco

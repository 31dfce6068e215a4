// bwd_rot.cuh -- adjoint of the all-pairs matrix from stored rotations (tcgen05 contraction only).
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// The forward can store each pair's optimal rotation R_ab (pairs_tc_kernel with ROT); then the
// adjoint needs no covariance and no rotation arithmetic: per tile it only gathers R_ab (or
// R_ba^T for the lower triangle), c_ab and w_ab, scales, and contracts. Same tiling as the
// recomputing adjoint (bwd_rc.cuh): a CTA owns one A tile I (40 models = 128 operand rows) and a contiguous range
// of B tiles J over the full square (every b != a in both orders, so no atomics on the
// gradient). Roles:
//   warp 0 (TMA): X_J^T hi / lo FP16 chunks (128 atoms x the tile's 64 operand rows) into a
//     2-stage ring;
//   warp 1 (MMA): the contraction transposed, sum^T += X_J^T . P_J^T (tcgen05 kind::f16 with
//     FP16 operands, M = 128 atoms, N = 128 rows of the A tile, K = 16, three passes
//     hi.hi + hi.lo + lo.hi). The accumulator holds ceil(Lp/128) blocks of 128 columns (TMEM
//     lanes = atoms);
//   warps 2-9 (epilogue): warp (sp, g) owns 10 A models x the 10 B models of half g of every
//     tile. Its gathers run one tile ahead through a 2-stage shared-memory ring: the rotation
//     records come as ten contiguous segments by bulk copy (in the condensed order the ten
//     records of a row, or of a column below the diagonal, are adjacent), c and w by 4-byte
//     asynchronous copies; warps whose block straddles the diagonal gather with plain loads.
//     Each lane then owns one row (model a, axis alpha) of the tile's 128 x 64 operand: row
//     alpha of w~ R_ab (or column alpha of R_ba), split into FP16 hi / lo parts and stored with
//     16-byte stores into one of two shared operands (128-byte swizzle, K-major), so that tile
//     J+1's operand is written while the MMAs read tile J's. Pairs below the near-duplicate
//     threshold go to the FP64 direct kernel, as in the recompute path.
// FP16 parts carry 22 significant bits, as TF32 hi / lo parts do, at twice the TF32 MMA rate.
// Both operands are scaled by powers of two so that their largest possible magnitude lies in
// [2^14, 2^15): X by the largest centred coordinate, the rotation operand by the bound
// max|w| / (L max(NEARDUP, eps)) on |w~| (|R_ij| <= 1); the readout undoes both exactly.
// At the end the CTA's sum goes out of TMEM into its partial slice; bwd_reduce_kernel adds the
// partials, the diagonal term and the centring projection.
#pragma once
#include <cuda_fp16.h>

#include <type_traits>

#include "bwd_tc.cuh"

namespace clusco {

constexpr int BR_THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int BR_XSTAGES = 2;
constexpr int BR_MAXLP = 512;
constexpr int BR_ABLK = 128;                     // atoms per accumulator block (MMA M)
constexpr uint32_t BR_A2 = 2 * 128 * 128;        // one operand: hi, lo parts of 128 rows x 64 FP16
constexpr uint32_t BR_XBUF = 2 * BR_ABLK * 128;  // one X^T chunk: hi, lo parts of 128 atoms x 64 FP16
constexpr uint32_t BR_SEG = 496;                 // one record segment: 10 x 48 B, padded against bank conflicts
constexpr uint32_t BR_RECW = 10 * BR_SEG;        // one warp's records of one tile
constexpr uint32_t BR_REC = 8 * BR_RECW;         // one stage of all eight epilogue warps
constexpr uint32_t BR_CWW = 200;                 // floats per warp and stage: c[10][10], w[10][10]
constexpr size_t BR_SMEM = 1024 + 2 * BR_A2 + BR_XSTAGES * BR_XBUF + 2 * BR_REC + 2 * 8 * BR_CWW * 4;
static_assert(BR_SMEM + 1024 <= 227 * 1024, "shared memory per CTA");

// k such that m 2^k lies in [2^14, 2^15) (0 when m is zero or not finite), clamped to +-100.
__host__ __device__ __forceinline__ int fp16_scale_exp(float m)
{
    if (!(m > 0.f) || !(m <= 3.0e38f)) return 0;
    int e;
    frexpf(m, &e);
    const int k = 15 - e;
    return k < -100 ? -100 : (k > 100 ? 100 : k);
}

__device__ __forceinline__ float exp2i(int k) { return __int_as_float((127 + k) << 23); }

// Centred FP32 rows in the tensor-core row layout (zero padding) and the largest |centred
// coordinate| over the finite models (atomicMax on the bits: they order like the values for
// x >= 0). Grid: ceil(Npad/8) blocks of 256 threads, one warp per model slot.
__global__ void __launch_bounds__(256) bwr_prepass_kernel(const float *__restrict__ coords, int64_t N, int L, int Lp,
                                                          int64_t Npad, float *__restrict__ xf,
                                                          unsigned *__restrict__ xmax)
{
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (a >= Npad) return;
    auto zero_row = [&](int64_t r) {
        for (int i = lane; i < Lp; i += 32) xf[r * Lp + i] = 0.f;
    };
    if (a % 10 == 9) {  // the two padding rows that close this model's 32-row group
        zero_row(32 * (a / 10) + 30);
        zero_row(32 * (a / 10) + 31);
    }
    const int64_t r0 = tc_row(a, 0);
    if (a >= N) {
        for (int ax = 0; ax < 3; ++ax) zero_row(r0 + ax);
        return;
    }
    const float *x = coords + a * (int64_t)L * 3;
    float mu[3];
    bool finite;
    model_centroid(x, L, lane, mu, &finite);
    float m = 0.f;
    for (int i = lane; i < Lp; i += 32)
        for (int ax = 0; ax < 3; ++ax) {
            const float v = (i < L) ? (x[3 * i + ax] - mu[ax]) : 0.f;
            xf[(r0 + ax) * Lp + i] = v;
            m = fmaxf(m, fabsf(v));
        }
    m = warp_max_f(m);
    if (lane == 0 && finite && m > 0.f) atomicMax(xmax, __float_as_uint(m));
}

// xT[part][i][r] = FP16 part (hi, lo) of xf[r][i] 2^kx, 32 x 32 tiles through shared memory.
__global__ void __launch_bounds__(256) bwr_split_kernel(const float *__restrict__ xf, int64_t Rpad, int Lp,
                                                        const unsigned *__restrict__ xmax, __half *__restrict__ xT)
{
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const float sx = exp2i(fp16_scale_exp(__uint_as_float(*xmax)));
    for (int k = ty; k < 32; k += 8) t[k][tx] = xf[(r0 + k) * Lp + i0 + tx];
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const float v = t[tx][k] * sx;
        const __half hi = __float2half_rn(v);
        xT[(int64_t)(i0 + k) * Rpad + r0 + tx] = hi;
        xT[((int64_t)Lp + i0 + k) * Rpad + r0 + tx] = __float2half_rn(v - __half2float(hi));
    }
}

// wmax = max |w| over the P weights (NaN ignored), 16-byte loads where w is 16-byte aligned.
__global__ void __launch_bounds__(256) bwr_absmax_kernel(const float *__restrict__ w, int64_t P,
                                                         unsigned *__restrict__ wmax)
{
    __shared__ float red[8];
    const int64_t nthr = (int64_t)gridDim.x * 256, tid = (int64_t)blockIdx.x * 256 + threadIdx.x;
    float m = 0.f;
    int64_t head = 0;
    if (((uintptr_t)w & 15) == 0) {
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        const int64_t n4 = P / 4;
        for (int64_t q = tid; q < n4; q += nthr) {
            const float4 v = __ldg(w4 + q);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        head = 4 * n4;
    }
    for (int64_t p = head + tid; p < P; p += nthr) m = fmaxf(m, fabsf(w[p]));
    m = warp_max_f(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) m = fmaxf(m, red[k]);
        if (m > 0.f) atomicMax(wmax, __float_as_uint(m));
    }
}

// Where a warp's 10 x 10 block of pairs lies: 0 all b > a (records along rows a), 1 all b < a
// (records along rows b), 2 straddling the diagonal.
__device__ __forceinline__ int br_mode(int64_t a0, int64_t b0) { return b0 > a0 + 9 ? 0 : (b0 + 9 < a0 ? 1 : 2); }

__global__ void __launch_bounds__(BR_THREADS, 1)
    bwd_rot_kernel(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl, int64_t N,
                   int L, int Lp, uint32_t tmem_cols, int64_t Rpad, int64_t TB, int64_t S, int64_t JC,
                   const float *__restrict__ crmsd, const float *__restrict__ wvec, const float *__restrict__ rot,
                   float eps, const unsigned *__restrict__ scl, float *__restrict__ Gp, float *__restrict__ dp,
                   long long *__restrict__ nd_list, unsigned long long *__restrict__ nd_count, int64_t nd_cap)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t xfull_bar[BR_XSTAGES];   // an X^T chunk landed
    __shared__ __align__(8) uint64_t xempty_bar[BR_XSTAGES];  // the MMAs have finished reading it
    __shared__ __align__(8) uint64_t a2full_bar[2];           // a rotation operand is written (8 arrivals)
    __shared__ __align__(8) uint64_t a2empty_bar[2];          // the MMAs have finished reading it
    __shared__ __align__(8) uint64_t d2_bar;                  // the last MMA has finished
    __shared__ __align__(8) uint64_t rec_bar[2][8];           // a warp's record segments landed
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float dsum[TC_MA];

    // 1024-byte aligned in the shared window; indexing smem_raw (not an integer cast) keeps the
    // pointer in the shared address space, so accesses through it compile to shared loads/stores
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *A2 = smem;                                       // two operands of BR_A2 bytes: [hi 16 KB][lo 16 KB]
    uint8_t *XT = smem + 2 * BR_A2;                           // BR_XSTAGES chunk buffers of BR_XBUF bytes
    uint8_t *REC = XT + BR_XSTAGES * BR_XBUF;                 // 2 stages x 8 warps x 10 segments
    float *CW = reinterpret_cast<float *>(REC + 2 * BR_REC);  // 2 stages x 8 warps x [c 100 | w 100]
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
            for (int w = 0; w < 8; ++w) mbar_init(&rec_bar[b][w], 1);
        }
        mbar_init(&d2_bar, 1);
        abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    // pad rows and columns of both operands stay zero for the whole sweep
    for (int e = tid; e < (int)(2 * BR_A2 / 16); e += BR_THREADS)
        reinterpret_cast<float4 *>(A2)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < TC_MA) dsum[tid] = 0.f;
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int64_t nJ = J1 - J0;
    const int nblk = (Lp + BR_ABLK - 1) / BR_ABLK;  // X^T chunks (atom blocks) per tile
    volatile int *abort_v = &abort_flag;
    int64_t xq = 0;  // X^T stages the producer (warp 0, lane 0) has armed

    if (warp == 0) {
        // ================= TMA producer: X^T chunks =================
        if (lane == 0) {
            int64_t &c = xq;
            bool ok = true;
            for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) {
                const int64_t J = J0 + j;
                for (int blk = 0; blk < nblk && ok; ++blk, ++c) {
                    const int st = (int)(c % BR_XSTAGES);
                    const int64_t use = c / BR_XSTAGES;
                    if (c >= BR_XSTAGES && !mbar_wait_sleep(&xempty_bar[st], (uint32_t)((use - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    // the tile's 64 operand rows x 128 atoms; atoms past Lp read zeros
                    const int x = (int)(64 * J), y = blk * BR_ABLK;
                    mbar_arrive_expect_tx(&xfull_bar[st], BR_XBUF);
                    tma_load_2d(XT + st * BR_XBUF, &mapXh, &xfull_bar[st], x, y);
                    tma_load_2d(XT + st * BR_XBUF + BR_XBUF / 2, &mapXl, &xfull_bar[st], x, y);
                }
            }
            if (!ok) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            int64_t c = 0;
            bool ok = true;
            constexpr uint32_t idesc = make_idesc(BR_ABLK, 128, 0);  // FP16 operands
            for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) {
                const int buf = (int)(j & 1);
                if (!mbar_wait_sleep(&a2full_bar[buf], (uint32_t)((j >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ab = a2base + (uint32_t)(buf * BR_A2);
                for (int blk = 0; blk < nblk && ok; ++blk, ++c) {
                    const int st = (int)(c % BR_XSTAGES);
                    if (!mbar_wait(&xfull_bar[st], (uint32_t)((c / BR_XSTAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xb = xtbase + st * BR_XBUF;
                    const uint32_t d = tmem + (uint32_t)(blk * 128);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        // A = X^T (atoms x operand rows), B = P (A-tile rows x operand rows), both
                        // K-major; K = 16 FP16 = 32 bytes per step along the swizzled rows
                        const uint64_t xhi = desc_sw128(xb + 32 * k);
                        const uint64_t xlo = desc_sw128(xb + BR_XBUF / 2 + 32 * k);
                        const uint64_t phi = desc_sw128(ab + 32 * k);
                        const uint64_t plo = desc_sw128(ab + BR_A2 / 2 + 32 * k);
                        // each block's first MMA of the sweep starts its columns from zero
                        mma_f16(d, xhi, phi, idesc, (j == 0 && k == 0) ? 0u : 1u);
                        mma_f16(d, xhi, plo, idesc, 1u);
                        mma_f16(d, xlo, phi, idesc, 1u);
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
        const int etid = tid - 64, ew = warp - 2;
        const int sp = warp & 3, g = ew >> 2;
        const int mloc = lane / 3, alpha = lane - 3 * (lane / 3);
        const int ml = lane < 30 ? mloc : 9;  // shared-memory row of the two pad lanes (never used)
        const int la = 10 * sp + mloc;
        const int64_t a0 = a_base + 10 * sp, a = a0 + mloc;
        const bool lane_ok = lane < 30 && a < N;
        const int na = (int)(N - a0 < 0 ? 0 : (N - a0 > 10 ? 10 : N - a0));
        const float fL = (float)L;
        const int kx = fp16_scale_exp(__uint_as_float(scl[0]));
        const int kp = fp16_scale_exp(__uint_as_float(scl[1]) / (fL * fmaxf(CLUSCO_NEARDUP, eps)));
        const float sP = exp2i(kp);

        // Gathers of tile jj into stage jj & 1 (the stage's previous tile, jj - 2, is consumed).
        auto issue = [&](int64_t jj) {
            const int s = (int)(jj & 1);
            const int64_t b0 = (J0 + jj) * TC_MB + 10 * g;
            const int mode = br_mode(a0, b0);
            const int nb = (int)(N - b0 < 0 ? 0 : (N - b0 > 10 ? 10 : N - b0));
            uint8_t *rw = REC + s * BR_REC + ew * BR_RECW;
            float *cw = CW + (s * 8 + ew) * BR_CWW;
            uint64_t *bar = &rec_bar[s][ew];
            if (mode == 2) {
                // straddles the diagonal: plain loads, stored as row alpha of the effective
                // rotation (R_ab, or R_ba^T when b < a) in the layout of mode 0
#pragma unroll 1
                for (int bq = 0; bq < 10; ++bq) {
                    const int64_t b = b0 + bq;
                    if (lane_ok && b < N && b != a) {
                        const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
                        const int64_t idx = condensed_idx(lo, hi, N);
                        const float *rec = rot + idx * ROT_STRIDE;
                        const int o0 = a < b ? 3 * alpha : alpha, st = a < b ? 1 : 3;
                        float *d = reinterpret_cast<float *>(rw + mloc * BR_SEG + bq * 48) + 3 * alpha;
                        d[0] = __ldg(rec + o0);
                        d[1] = __ldg(rec + o0 + st);
                        d[2] = __ldg(rec + o0 + 2 * st);
                        if (alpha < 2) cp_async4(cw + alpha * 100 + mloc * 10 + bq, (alpha ? wvec : crmsd) + idx);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(bar);
            } else {
                // ten contiguous segments: rows a0.. (records b0..b0+nb-1) above the diagonal,
                // rows b0.. (records a0..a0+na-1) below it
                const int nseg = mode == 0 ? na : nb, nrec = mode == 0 ? nb : na;
                fence_proxy_async();  // earlier generic accesses of the stage before the async writes
                if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(48 * nseg * nrec));
                __syncwarp();
                if (lane < nseg && nrec > 0) {
                    const int64_t idx = mode == 0 ? condensed_idx(a0 + lane, b0, N) : condensed_idx(b0 + lane, a0, N);
                    bulk_load(rw + lane * BR_SEG, rot + idx * ROT_STRIDE, (uint32_t)(48 * nrec), bar);
                }
                if (lane_ok && alpha < 2) {  // c (alpha 0) or w (alpha 1) of this lane's model row
                    const float *src = alpha ? wvec : crmsd;
                    float *d = cw + alpha * 100 + mloc * 10;
                    if (mode == 0) {
                        const float *s0 = src + condensed_idx(a, b0, N);
#pragma unroll
                        for (int bq = 0; bq < 10; ++bq)
                            if (bq < nb) cp_async4(d + bq, s0 + bq);
                    } else {
                        // idx(b + 1, a) = idx(b, a) + N - b - 2
                        const float *s0 = src + condensed_idx(b0, a, N);
                        const int64_t step0 = N - b0 - 2;
#pragma unroll
                        for (int bq = 0; bq < 10; ++bq)
                            if (bq < nb) cp_async4(d + bq, s0 + (bq * step0 - (int64_t)(bq * (bq - 1) / 2)));
                    }
                }
            }
            cp_async_commit();
        };

        bool alive = true;
        int64_t jfail = -1;  // the tile being processed when the sweep was abandoned
        issue(0);
        for (int64_t j = 0; j < nJ; ++j) {
            const int buf = (int)(j & 1);
            if (j + 1 < nJ) issue(j + 1);
            bool ok = mbar_wait_sleep(&rec_bar[buf][ew], (uint32_t)((j >> 1) & 1));
            if (j + 1 < nJ)
                cp_async_wait<1>();
            else
                cp_async_wait<0>();
            __syncwarp();
            const int64_t b0 = (J0 + j) * TC_MB + 10 * g;
            const int mode = br_mode(a0, b0);
            const uint8_t *rw = REC + buf * BR_REC + ew * BR_RECW;
            const float *cw = CW + (buf * 8 + ew) * BR_CWW;
            // pair (a, b0 + bq) is valid for bq < nbv, bq != self (b == a only straddling the diagonal)
            const int nbv = lane_ok ? (int)(N - b0 < 0 ? 0 : (N - b0 > 10 ? 10 : N - b0)) : 0;
            const int self = (int)(a - b0);
            float v[32];
            float csum = 0.f;
            uint32_t ndm = 0;  // pairs below the near-duplicate threshold, queued after the loop
            // One straight-line pass over the ten B models: row alpha of R_ab from record (a, b)
            // along row a (mode 0, and the diagonal blocks' gathered rows), or column alpha of
            // R_ba from record (b, a) along row b (mode 1).
            auto consume = [&](auto below) {
                constexpr bool M1 = decltype(below)::value;
#pragma unroll
                for (int bq = 0; bq < 10; ++bq) {
                    const bool valid = bq < nbv && bq != self;
                    const float c = cw[ml * 10 + bq], w = cw[100 + ml * 10 + bq];
                    const float *r = M1 ? reinterpret_cast<const float *>(rw + bq * BR_SEG + ml * 48) + alpha
                                        : reinterpret_cast<const float *>(rw + ml * BR_SEG + bq * 48) + 3 * alpha;
                    constexpr int st = M1 ? 3 : 1;
                    const float r0 = r[0], r1 = r[st], r2 = r[2 * st];
                    const bool far = c >= CLUSCO_NEARDUP;
                    ndm |= (valid && !far && w != 0.f) ? (1u << bq) : 0u;
                    const float coef = (valid && far) ? __fdividef(w, fL * fmaxf(c, eps)) : 0.f;
                    csum += coef;
                    const float cs = coef * sP;
                    v[3 * bq + 0] = valid ? cs * r0 : 0.f;
                    v[3 * bq + 1] = valid ? cs * r1 : 0.f;
                    v[3 * bq + 2] = valid ? cs * r2 : 0.f;
                }
            };
            if (mode == 1)
                consume(std::true_type{});
            else
                consume(std::false_type{});
            if (ndm != 0u && alpha == 0) {  // rare: one lane per pair queues it, from the a < b side
                for (int bq = 0; bq < 10; ++bq) {
                    const int64_t b = b0 + bq;
                    if (((ndm >> bq) & 1u) && a < b) {
                        const unsigned long long slot = atomicAdd(nd_count, 1ull);
                        if ((int64_t)slot < nd_cap) {
                            nd_list[2 * slot] = a;
                            nd_list[2 * slot + 1] = b;
                        }
                    }
                }
            }
            v[30] = v[31] = 0.f;
            if (alpha == 0 && lane_ok) atomicAdd(&dsum[la], csum);
            // the operand buffer is reused every other tile: wait until the MMAs of tile j-2 read it
            if (j >= 2) ok = mbar_wait_sleep(&a2empty_bar[buf], (uint32_t)(((j >> 1) - 1) & 1)) && ok;
            // each warp decides for itself (no barrier per tile); a warp that stops raises the
            // flag, and the others' bounded waits end their sweeps
            if (__any_sync(0xffffffffu, !ok || *abort_v)) {
                if (lane == 0) atomicExch(&abort_flag, 1);
                alive = false;
                jfail = j;
                break;
            }
            // the row, as FP16 hi / lo parts, into the 128-byte-swizzled K-major operand: row
            // 32 sp + lane, half g of its 128 bytes = four 16-byte chunks at (chunk ^ (row mod 8))
            if (lane < 30) {
                const int row = 32 * sp + lane;
                uint8_t *base = A2 + buf * BR_A2 + row * 128;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float x0 = v[8 * q + 2 * e], x1 = v[8 * q + 2 * e + 1];
                        const __half2 hh = __floats2half2_rn(x0, x1);
                        const float2 hf = __half22float2(hh);
                        const __half2 ll = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
                        h[e] = *reinterpret_cast<const uint32_t *>(&hh);
                        l[e] = *reinterpret_cast<const uint32_t *>(&ll);
                    }
                    const int off = (((4 * g + q) ^ (row & 7)) & 7) << 4;
                    *reinterpret_cast<uint4 *>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(base + BR_A2 / 2 + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_proxy_async();  // generic-proxy stores to the operand must be visible to tcgen05.mma
            __syncwarp();
            if (lane == 0) mbar_arrive(&a2full_bar[buf]);
        }
        if (!alive) {
            // the gathers of the abandoned tile and of the next one may still be in flight: let
            // them land (bounded) before the CTA's shared memory goes away
            mbar_wait(&rec_bar[jfail & 1][ew], (uint32_t)((jfail >> 1) & 1));
            if (jfail + 1 < nJ) mbar_wait(&rec_bar[(jfail + 1) & 1][ew], (uint32_t)(((jfail + 1) >> 1) & 1));
            cp_async_wait<0>();
        }
        {  // every epilogue warp, stopped or not, meets the others here once
            const bool ok3 = alive && mbar_wait_sleep(&d2_bar, 0);
            alive = !named_bar_or(1, 256, !ok3 || *abort_v);
        }
        if (alive) {
            tc_fence_after();
            // read the transposed sum out of TMEM: warp (sp, g) takes TMEM lanes 32 sp.. (atoms)
            // and half g of each block's 128 columns (rows of the A tile); undo both scales
            const float ix = exp2i(-kx), ip = exp2i(-kp);
            float *gbase = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
            for (int blk = 0; blk < nblk; ++blk) {
                const int atom = blk * BR_ABLK + 32 * sp + lane;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r0 = 64 * g + 32 * h;
                    float vv[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)(blk * 128 + r0), vv);
                    if (atom < Lp) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) gbase[(int64_t)(r0 + jj) * Lp + atom] = -(vv[jj] * ix) * ip;
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
    if (warp == 0) {
        if (lane == 0 && *abort_v) {
            // a stopped CTA: the copies of the last armed stages may still be in flight (the MMA
            // issuer stopped waiting for them); they land before the CTA leaves (bounded waits)
            for (int64_t r = (xq > BR_XSTAGES ? xq - BR_XSTAGES : 0); r < xq; ++r)
                mbar_wait(&xfull_bar[r % BR_XSTAGES], (uint32_t)((r / BR_XSTAGES) & 1));
        }
        __syncwarp();
        tmem_dealloc(tmem, tmem_cols);
    }
}

inline bool bwr_supported(int64_t L) { return (L + 63) / 64 * 64 <= BR_MAXLP; }

// Host side, in two parts. bwr_prepare: the pre-pass (centred FP32 rows, transposed FP16
// parts, the two scales), which reads only the coordinates and the weights, so that it may run
// beside the forward. bwr_sweep: the contraction sweep from stored rotations, the reduction and
// the FP64 near-duplicate kernel, after the forward and the pre-pass. Workspace: carve_bt's
// layout (its TF32 transpose buffer holds the FP16 parts here).
inline int bwr_prepare(const float *coords, int64_t N, int64_t L, const float *grad_out, void *ws, cudaStream_t st,
                       std::string &err)
{
    const BtWs w = carve_bt(ws, N, L);
    const int64_t P = N * (N - 1) / 2;
    __half *xT = reinterpret_cast<__half *>(w.xT);
    cudaError_t e = cudaMemsetAsync(w.scl, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.nd_count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        bwr_prepass_kernel<<<(unsigned)((w.Npad + 7) / 8), 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.xf,
                                                                         w.scl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bwr_split_kernel<<<dim3((unsigned)(w.Rpad / 32), (unsigned)(w.Lp / 32)), 256, 0, st>>>(w.xf, w.Rpad, (int)w.Lp,
                                                                                              w.scl, xT);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bwr_absmax_kernel<<<4 * 148, 256, 0, st>>>(grad_out, P, w.scl + 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("backward pre-pass: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

inline int bwr_sweep(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                     const float *rot, float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
{
    const BtWs w = carve_bt(ws, N, L);
    __half *xT = reinterpret_cast<__half *>(w.xT);
    cudaError_t e = cudaSuccess;
    CUtensorMap mXh, mXl;
    for (int part = 0; part < 2; ++part) {
        // X^T hi / lo parts: FP16 [Lp][Rpad] each; boxes of the tile's 64 operand rows (128
        // bytes) x 128 atoms; atoms past Lp read as zeros
        const cuuint64_t dims[2] = {(cuuint64_t)w.Rpad, (cuuint64_t)w.Lp};
        const cuuint64_t strides[1] = {(cuuint64_t)(w.Rpad * 2)};
        const cuuint32_t box[2] = {64u, (cuuint32_t)BR_ABLK};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(part ? &mXl : &mXh, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, xT + part * w.Lp * w.Rpad,
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
        bwd_rot_kernel<<<grid, BR_THREADS, BR_SMEM, st>>>(mXh, mXl, N, (int)L, (int)w.Lp, cols, w.Rpad, TB, w.S, JC,
                                                          crmsd, grad_out, rot, eps, w.scl, w.Gp, w.dp, w.nd_list,
                                                          w.nd_count, w.nd_cap);
        e = cudaGetLastError();
        prof_mark(PROF_ADJOINT, st);
    }
    if (e == cudaSuccess) {
        e = launch_bwd_reduce(w, N, L, grad, st);
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

inline int bwr_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                      const float *rot, float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
{
    const int rc = bwr_prepare(coords, N, L, grad_out, ws, st, err);
    return rc ? rc : bwr_sweep(coords, N, L, grad_out, crmsd, rot, grad, eps, ws, st, err);
}

}  // namespace clusco

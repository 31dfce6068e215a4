// pairs_tc.cuh -- tensor-core (tcgen05) all-pairs cRMSD: the covariance stage of eq. 2
// as the contraction X X^T over K = L atoms, fused with the per-pair eq. 2 epilogue.
//
// Operands (written by prepass_tc_kernel): K-contiguous planes of 3N rows, rows grouped
// 32 at a time as 10 models x 3 axes + 2 zero rows. One CTA computes one tile of
// 40 A-models (128 rows) x 20 B-models (64 rows): the 128 x N block of X_A X_B^T holds
// the 3x3 covariance blocks of its 800 model pairs. Only tiles with pairs a < b exist
// (upper triangle: B-tile J >= 2 I).
//
// Pipeline (persistent: one CTA per SM, CTA x takes tiles x, x + grid, ...; 10 warps, or 18
// with the 5-model windows below): warp 0 lane 0 streams 64-column K blocks of the A and B
// tiles into a 3-stage shared-memory ring with TMA (128-byte swizzle); warp 1 lane 0 issues
// tcgen05.mma into one of two 256-column TMEM accumulator buffers, so that the MMAs of tile
// k + 1 run while the epilogue warps (8, or 16 on windows) drain tile k: tcgen05.ld of their
// 32 TMEM lanes and columns, assembly of each 3x3 block across the three lanes of a model with
// warp shuffles, eq. 2 in the normalised frame, condensed FP32 store (or the threshold list).
// No covariance reaches global memory.
//
// Forms:
//  EXACT2: planes h, l of 16-bit fixed point (n = 256 h + l). Per 16-wide K step two
//    MMAs of N = 128 against B' = [B_h; B_l]: A_h B'^T -> TMEM cols [0,128) (hh | hl),
//    A_l B'^T -> cols [128,256) (lh | ll). Four digit-product classes, each an exact
//    integer sum in FP32 (|digit| <= 128, L <= 1024 keeps every sum below 2^24).
//    Epilogue: FP32 fast path; pairs whose FP32 error bound exceeds the fast-path
//    tolerance go to their epilogue warp's list (past its capacity: a bit in a mask) and are
//    recomputed after the sweep, exactly from the 16-bit coordinates and in FP64
//    (refine_flagged_kernel).
//  BF16X3: planes hi, lo; A_h B'^T (hh | hl) and A_l B_h^T (lh); H = hh + hl + lh.
//  TF32: one FP32 plane; A B^T with kind::tf32.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "epilogue.cuh"
#include "prepass.cuh"
#include "prof.cuh"
#include "ptx.cuh"
#include "rotation.cuh"

#ifndef CLUSCO_TOL_FAST
#define CLUSCO_TOL_FAST 5e-4f  // A: largest FP32 fast-path error accepted for the exact form
#endif

namespace clusco {

// Stored rotations: one 48-byte record per pair, R_ab row-major in floats 0..8 and zeros in
// 9..11, so that it moves as three 16-byte vectors.
constexpr int ROT_STRIDE = 12;

__device__ __forceinline__ void store_rot(float *dst, const float R[9])
{
    float4 *d = reinterpret_cast<float4 *>(dst);
    d[0] = make_float4(R[0], R[1], R[2], R[3]);
    d[1] = make_float4(R[4], R[5], R[6], R[7]);
    d[2] = make_float4(R[8], 0.f, 0.f, 0.f);
}

// A pair whose rotation the closed form cannot give accurately (P' below 0.08 Sigma^3, about
// 0.5 % of the pairs of a decoy ensemble): the forward appends its normalised covariance
// (natural axis order) and rot_fixup_kernel solves it by Jacobi sweeps afterwards, one pair per
// thread, instead of a divergent slow path inside the epilogue's rounds.
struct RotFix {
    long long idx;  // condensed index relative to the output's base
    float m[9];
    float pad;
};
static_assert(sizeof(RotFix) == 48, "deferred rotation entry");

struct TcArgs {
    int form;
    void *planes;
    float *scales;
    double *G64;
    float *G32;
    int64_t N, L, Lp, Rpad, row_begin, row_end;
    float *out;
    int64_t out_base;
    float *rot = nullptr;  // optional: R_ab per pair, [P][ROT_STRIDE] in the output's condensed order
    RotFix *fix = nullptr;            // deferred rotations (see RotFix)
    unsigned long long *fix_count = nullptr;
    int64_t fix_cap = 0;
    uint32_t *flags = nullptr;  // EXACT2: one bit per output pair (flagged pairs past a warp's list),
                                // then FL_MAXSLOTS list counts (flag_list_offset)
    int2 *flist = nullptr;      // EXACT2: the flagged pairs (a, b), one list per epilogue warp
    int64_t flist_entries = 0;  // capacity of flist over all warps
    int8_t *hplane = nullptr;   // EXACT2: the 16-bit fixed-point coordinates as bytes (h, l), for
    int8_t *lplane = nullptr;   // the refinement of flagged pairs
    // threshold mode (list != nullptr; no rotations): the pairs with c < tau instead of out
    long long *list = nullptr;
    float *vals = nullptr;
    unsigned long long *count = nullptr;
    int64_t cap = 0;
    float tau = 0.f;
};



constexpr uint32_t STAGE_BYTES_BF16 = 2 * 16384 + 2 * 8192;  // A_h, A_l, B_h, B_l
constexpr uint32_t STAGE_BYTES_TF32 = 16384 + 8192;          // A, B
// Persistent forward kernel: 1 CTA per SM, warp 0 TMA, warp 1 MMA, then the epilogue warps:
// with WIN 16 (four per TMEM lane quadrant, each the quadrant's 10 A models against a 5-model
// window of the tile's 20 B models), else 8 (two per quadrant, 10-model halves).
__host__ __device__ constexpr int fw_epi(bool win) { return win ? 16 : 8; }
__host__ __device__ constexpr int fw_threads(bool win) { return 64 + 32 * fw_epi(win); }
// the 5-model windows pay off while the epilogue alone bounds the kernel; with more atoms per
// pair the MMA stream takes a larger share and the extra warps cost more than they give
// (0.495 -> 0.434 ms at 5,000 x 300, 1.734 -> 1.770 ms at 8,192 x 500 for the forward call)
constexpr int64_t FW_WIN_MAXLP = 384;
constexpr int FW_MAXEPI = 16;
constexpr int FW_STAGES = 3;
// threshold mode: per epilogue warp, a staging buffer of 64 kept pairs (global index, value),
// published 32 at a time with one atomic
constexpr int FW_SBUF = 64;
constexpr size_t FW_SMEM = 1024 + FW_STAGES * STAGE_BYTES_BF16 + FW_MAXEPI * FW_SBUF * 12;
static_assert(FW_SMEM <= 227 * 1024, "shared memory per CTA");

__host__ __device__ __forceinline__ int64_t tc_row_start(int64_t I, int64_t TB) { return I * TB - I * (I - 1); }

// Tile t -> (I, J): rows I in order, J in [2I, TB).
__device__ __forceinline__ void tc_decode(int64_t t, int64_t TB, int64_t TA, int64_t *I, int64_t *J)
{
    const double b = (double)TB + 1.0;
    int64_t i = (int64_t)floor((b - sqrt(fmax(b * b - 4.0 * (double)t, 0.0))) * 0.5);
    if (i < 0) i = 0;
    if (i > TA - 1) i = TA - 1;
    while (i > 0 && tc_row_start(i, TB) > t) --i;
    while (i + 1 < TA && tc_row_start(i + 1, TB) <= t) ++i;
    *I = i;
    *J = 2 * i + (t - tc_row_start(i, TB));
}

// Advance (I, J) by `step` tiles in the row-major order of the upper-triangle tiles (row I
// holds J = 2I .. TB-1): integer carries only, no square root after the first decode.
__device__ __forceinline__ void tc_advance(int64_t &I, int64_t &J, int64_t step, int64_t TB, int64_t TA)
{
    J += step;
    while (J >= TB && I + 1 < TA) {
        J -= TB;
        ++I;
        J += 2 * I;
    }
}

template <int LAYOUT>
__device__ __forceinline__ void tc_issue_kblock(uint32_t tmem, uint32_t sbase, int kb)
{
    if (LAYOUT == TC_TF32) {
        constexpr uint32_t id = make_idesc(128, 64, 2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t a = desc_sw128(sbase + 32 * k);
            const uint64_t b = desc_sw128(sbase + 16384 + 32 * k);
            mma_tf32(tmem, a, b, id, (kb > 0 || k > 0) ? 1u : 0u);
        }
    } else {
        constexpr uint32_t id128 = make_idesc(128, 128, 1);
        constexpr uint32_t id64 = make_idesc(128, 64, 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
            const uint64_t ah = desc_sw128(sbase + 32 * k);
            const uint64_t al = desc_sw128(sbase + 16384 + 32 * k);
            const uint64_t bb = desc_sw128(sbase + 32768 + 32 * k);  // [B_h; B_l], 128 rows
            mma_bf16(tmem + 0, ah, bb, id128, acc);
            if (LAYOUT == TC_EXACT2)
                mma_bf16(tmem + 128, al, bb, id128, acc);
            else
                mma_bf16(tmem + 128, al, bb, id64, acc);  // B_h only: lh
        }
    }
}

// Selection among three values by a small runtime index (no local memory).
__device__ __forceinline__ float sel3(int i, float a, float b, float c) { return i == 0 ? a : (i == 1 ? b : c); }

// Block assembly for round r (0..3). Lane (mloc, alpha) holds row alpha of model mloc's
// 3 x 32 strip (3 x 3 blocks of B models 0..9 at columns 3 b' + beta, plus 2 pad columns).
// In round r it gathers the whole block of B model 3 r + alpha: its own row from column
// group alpha and the two other rows by shuffles from the model's other two lanes, in the
// cyclic row order alpha, alpha + 1, alpha + 2 (a proper rotation of the rows, which
// leaves eq. 2 unchanged).
__device__ __forceinline__ void assemble_from_cand(const float (&cand)[3][3], int alpha, int mloc, float blk[9])
{
#pragma unroll
    for (int be = 0; be < 3; ++be) blk[be] = sel3(alpha, cand[0][be], cand[1][be], cand[2][be]);
#pragma unroll
    for (int kk = 1; kk <= 2; ++kk) {
        const int sendsel = (alpha + 3 - kk) % 3;
        const int src = 3 * mloc + (alpha + kk) % 3;
#pragma unroll
        for (int be = 0; be < 3; ++be)
            blk[3 * kk + be] = __shfl_sync(0xffffffffu, sel3(sendsel, cand[0][be], cand[1][be], cand[2][be]), src & 31);
    }
}

__device__ __forceinline__ void assemble_block(const float V[32], int r, int alpha, int mloc, float blk[9])
{
    float cand[3][3];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const int j = 9 * r + 3 * al + be;
            cand[al][be] = (j < 32) ? V[j] : 0.f;
        }
    assemble_from_cand(cand, alpha, mloc, blk);
}

// The 15 TMEM columns of a 5-model window of one warp's 32-column half (window 0: columns
// 0..14, window 1: 15..29 of the half, starting at taddr), one region (digit class) of the
// accumulator: window 1 takes one column and the 16 from column 16.
__device__ __forceinline__ void ld_window(uint32_t taddr, int hw, float (&w)[15])
{
    uint32_t u[16];
    if (hw == 0) {
        tmem_ld16_issue(taddr, u);
        tmem_wait_ld();
        tmem_pin16(u);
#pragma unroll
        for (int j = 0; j < 15; ++j) w[j] = __uint_as_float(u[j]);
    } else {
        uint32_t e = tmem_ld1_issue(taddr + 15);
        tmem_ld16_issue(taddr + 16, u);
        tmem_wait_ld();
        asm volatile("" : "+r"(e));
        tmem_pin16(u);
        w[0] = __uint_as_float(e);
#pragma unroll
        for (int j = 0; j < 14; ++j) w[j + 1] = __uint_as_float(u[j]);
    }
}

// assemble_block on a 5-model window (15 columns): round r holds window models 3 r + t; a lane
// whose model falls past the window gets a zero block (and has no pair).
template <int r>
__device__ __forceinline__ void assemble_window(const float (&V)[15], int alpha, int mloc, float blk[9])
{
    float cand[3][3];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const int j = 9 * r + 3 * al + be;
            cand[al][be] = (j < 15) ? V[j] : 0.f;
        }
    assemble_from_cand(cand, alpha, mloc, blk);
}

// The rotation of a rare block whose quartic root is (nearly) double (out of line): Jacobi
// sweeps for a rank-deficient block (I2 ~ 0, where an FP32 Sigma is least accurate), else
// Horn's adjugate with the block's Sigma, and Jacobi sweeps where that is degenerate too.
// (By value: an address taken in the caller would keep its matrices in local memory on every
// pass of the fast path, not only on the rare call.)
struct Mat3 {
    float e[9];
};

__device__ __noinline__ Mat3 rotation_robust_ool(Mat3 Hn)
{
    float Rl[9];
    float I1, det, I2;
    invariants3(Hn.e, I1, det, I2);
    if (!(I2 > 1e-8f * I1 * I1) || !horn_rotation(Hn.e, sigma_hat_f32(Hn.e), 1e-5f, Rl))
        rotation_jacobi4<float, 8>(Hn.e, Rl);
    Mat3 R;
#pragma unroll
    for (int e = 0; e < 9; ++e) R.e[e] = Rl[e];
    return R;
}

// Pointer form, for callers whose matrices already live in memory or whose registers are
// scarcer than their stack (the recompute adjoint).
__device__ __noinline__ void rotation_robust_ptr(const float *Hn, float *R)
{
    float Rl[9];
    float H[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) H[e] = Hn[e];
    float I1, det, I2;
    invariants3(H, I1, det, I2);
    if (!(I2 > 1e-8f * I1 * I1) || !horn_rotation(H, sigma_hat_f32(H), 1e-5f, Rl)) rotation_jacobi4<float, 8>(H, Rl);
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e] = Rl[e];
}

__device__ __forceinline__ void rotation_robust(const float Hn[9], float R[9])
{
    Mat3 h;
#pragma unroll
    for (int e = 0; e < 9; ++e) h.e[e] = Hn[e];
    const Mat3 r = rotation_robust_ool(h);
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e] = r.e[e];
}

// Deferred rotations: Jacobi sweeps on each listed pair's covariance (one pair per thread).
__global__ void __launch_bounds__(256) rot_fixup_kernel(const RotFix *__restrict__ list,
                                                        const unsigned long long *__restrict__ count, int64_t cap,
                                                        float *__restrict__ rot)
{
    const int64_t n = (int64_t)*count < cap ? (int64_t)*count : cap;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float m[9], R[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = list[i].m[e];
        rotation_jacobi4<float, 8>(m, R);
        store_rot(rot + list[i].idx * ROT_STRIDE, R);
    }
}

// ROT: also write each pair's optimal rotation R_ab (b onto a, natural axis order, row-major)
// to rot[(idx - out_base) * ROT_STRIDE ..], computed as dSigma/dM from the fast path's Sigma (Horn's
// key matrix near a double root); the adjoint reads it instead of recomputing the covariance.
template <int LAYOUT, bool ROT, bool SPARSE = false, bool WIN = false>
__global__ void __launch_bounds__(fw_threads(WIN), 1)
    pairs_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const float *__restrict__ scales, const float *__restrict__ G32,
                    int64_t N, int L, int nkb, int64_t Rpad, int64_t TA, int64_t TB, int64_t tile0, int64_t ntiles,
                    int64_t row_begin, int64_t row_end, PairSink sink,
                    float *__restrict__ rot, RotFix *__restrict__ fix, unsigned long long *__restrict__ fix_count,
                    int64_t fix_cap, uint32_t *__restrict__ flags, int2 *__restrict__ flist,
                    unsigned *__restrict__ fl_cnt, int fl_cap)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[FW_STAGES];   // ring: K block landed
    __shared__ __align__(8) uint64_t empty_bar[FW_STAGES];  // ring: K block consumed by the MMAs
    __shared__ __align__(8) uint64_t tfull_bar[2];          // accumulator buffer holds a finished tile
    __shared__ __align__(8) uint64_t tempty_bar[2];         // the epilogue has drained the buffer (one arrival per epilogue warp)
    __shared__ __align__(8) uint64_t done_bar;              // every MMA this CTA issued has completed
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    // 1024-byte aligned in the shared window; indexing smem_raw (not an integer cast) keeps the
    // pointer in the shared address space, so accesses through it compile to shared loads/stores
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase0 = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t STAGE_BYTES = (LAYOUT == TC_TF32) ? STAGE_BYTES_TF32 : STAGE_BYTES_BF16;
    constexpr int KB_ELEMS = (LAYOUT == TC_TF32) ? 32 : 64;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < FW_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], fw_epi(WIN));
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abort_v = &abort_flag;
    int64_t q = 0;  // stages the producer (warp 0, lane 0) has armed

    if (warp == 0) {
        // ================= TMA producer =================
        if (lane == 0) {
            tma_prefetch_desc(&mapA);
            tma_prefetch_desc(&mapB);
            int64_t I, J;
            tc_decode(tile0 + blockIdx.x, TB, TA, &I, &J);
            for (int64_t t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x, tc_advance(I, J, gridDim.x, TB, TA)) {
                for (int kb = 0; kb < nkb; ++kb, ++q) {
                    const int s = (int)(q % FW_STAGES);
                    const int64_t use = q / FW_STAGES;
                    if (q >= FW_STAGES && !mbar_wait_sleep(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                        atomicExch(&abort_flag, 1);
                        break;
                    }
#ifdef CLUSCO_DEBUG_HOOKS
                    if (g_debug_skip_arrive && blockIdx.x == 0 && q == 0) continue;  // stage 0 never lands
#endif
                    uint8_t *st = smem + s * STAGE_BYTES_BF16;
                    mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
                    const int x = kb * KB_ELEMS;
                    if (LAYOUT == TC_TF32) {
                        tma_load_2d(st, &mapA, &full_bar[s], x, (int)(128 * I));
                        tma_load_2d(st + 16384, &mapB, &full_bar[s], x, (int)(64 * J));
                    } else {
                        tma_load_2d(st, &mapA, &full_bar[s], x, (int)(128 * I));
                        tma_load_2d(st + 16384, &mapA, &full_bar[s], x, (int)(Rpad + 128 * I));
                        tma_load_2d(st + 32768, &mapB, &full_bar[s], x, (int)(64 * J));
                        tma_load_2d(st + 40960, &mapB, &full_bar[s], x, (int)(Rpad + 64 * J));
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            int64_t q = 0, k = 0;
            for (int64_t t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x, ++k) {
                const int buf = (int)(k & 1);
                const int64_t u = k >> 1;
                if (k >= 2 && !mbar_wait_sleep(&tempty_bar[buf], (uint32_t)((u - 1) & 1))) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                tc_fence_after();
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++q) {
                    const int s = (int)(q % FW_STAGES);
                    const int64_t use = q / FW_STAGES;
                    if (!mbar_wait_sleep(&full_bar[s], (uint32_t)(use & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    tc_issue_kblock<LAYOUT>(tmem + 256u * buf, sbase0 + s * STAGE_BYTES_BF16, kb);
                    mma_commit(&empty_bar[s]);
                }
                mma_commit(&tfull_bar[buf]);
                if (!ok) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
            }
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0)) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else {
        // ================= epilogue warps 2.. =================
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its lane quadrant, the 10 A models of its
        // rows); with rotations it takes column half g (10 B models), without them the 5-model
        // window hw of that half (columns 32 g + 15 hw .. + 14)
        const int ew = warp - 2;
        const int sp = warp & 3, g = (ew >> 2) & 1, hw = WIN ? (ew >> 3) : 0;
        const int mloc = lane / 3, alpha = lane - 3 * (lane / 3);
        const float invL = 1.f / (float)L;
        float *const out = sink.out;
        const int64_t out_base = sink.out_base;
        // threshold mode: this warp's staging buffer of kept pairs (fill is warp-uniform)
        long long *sidx = reinterpret_cast<long long *>(smem + FW_STAGES * STAGE_BYTES_BF16) + ew * FW_SBUF;
        float *sval = reinterpret_cast<float *>(smem + FW_STAGES * STAGE_BYTES_BF16 + 8 * FW_MAXEPI * FW_SBUF) +
                      ew * FW_SBUF;
        int fill = 0;
        // EXACT2: this warp's list of flagged pairs (a, b); the ones past its capacity set their
        // mask bit instead
        int nfl = 0;
        int2 *const myfl = flist ? flist + ((int64_t)blockIdx.x * fw_epi(WIN) + ew) * fl_cap : nullptr;
        auto publish = [&](int n) {  // the first n staged pairs to the list, one atomic
            __syncwarp();
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(sink.count, (unsigned long long)n);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (lane < n && base + lane < (unsigned long long)sink.cap) {
                sink.list[base + lane] = sidx[lane];
                sink.vals[base + lane] = sval[lane];
            }
            __syncwarp();
        };

        // one pair's result (li: its condensed index relative to the output's base): flag it for the
        // refinement, or store it (dense) / stage it (threshold)
        auto emit_pair = [&](float cv, float ev, bool pk, float Ga, float gbh, int64_t li, int64_t ia, int64_t ib) {
            const bool flagged = LAYOUT == TC_EXACT2 && pk && !(ev <= 2.f * CLUSCO_TOL_FAST * cv);
            const float cfin = (isnan(Ga) || isnan(gbh)) ? __int_as_float(0x7fc00000) : cv;
            if constexpr (LAYOUT == TC_EXACT2) {
                // the bound fails: refine_flagged_kernel writes (or keeps) this pair's value
                const unsigned fm = __ballot_sync(0xffffffffu, flagged);
                if (fm) {
                    const int pos = nfl + __popc(fm & ((1u << lane) - 1u));
                    if (flagged) {
                        if (pos < fl_cap)
                            myfl[pos] = make_int2((int)ia, (int)ib);
                        else
                            atomicOr(flags + (li >> 5), 1u << (li & 31));
                    }
                    nfl += __popc(fm);
                }
            }
            if (!flagged && !SPARSE && pk) out[li] = cfin;
            if (SPARSE) {
                const bool keep = pk && !flagged && cfin < sink.tau;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (m) {
                    if (keep) {
                        const int my = fill + __popc(m & ((1u << lane) - 1u));
                        sidx[my] = li + out_base;
                        sval[my] = cfin;
                    }
                    fill += __popc(m);
                    if (fill >= 32) {
                        publish(32);
                        if (lane < fill - 32) {
                            sidx[lane] = sidx[32 + lane];
                            sval[lane] = sval[32 + lane];
                        }
                        __syncwarp();
                        fill -= 32;
                    }
                }
            }
        };

        const int64_t gstep = gridDim.x;
        int64_t k = 0;
        int64_t I, J;
        tc_decode(tile0 + blockIdx.x, TB, TA, &I, &J);
        for (int64_t t = blockIdx.x; t < ntiles; t += gstep, ++k, tc_advance(I, J, gstep, TB, TA)) {
            if constexpr (WIN) {
                // the window: B models J TC_MB + 10 g + 5 hw + t (rounds 0, 1: t = alpha, 3 + alpha)
                const int64_t a = I * TC_MA + 10 * sp + mloc;
                const int64_t b0 = J * TC_MB + 10 * g + 5 * hw + alpha;
                const bool lane_ok = lane < 30 && a < N && a >= row_begin && a < row_end;
                const int64_t rowbase = a * N - a * (a + 1) / 2 - a - 1 - out_base;  // condensed index - b
                float srow0 = 1.f, Ga = 0.f;
                if (lane_ok) {
                    srow0 = scales[a * 3 + alpha];
                    Ga = G32[a];
                }
                bool pok[2];
                float Gb[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int64_t b = b0 + 3 * r;
                    pok[r] = lane_ok && (3 * r + alpha) < 5 && b < N && a < b;
                    Gb[r] = pok[r] ? __ldg(G32 + b) : 0.f;
                }
                const int buf = (int)(k & 1);
                const bool okw = mbar_wait_sleep(&tfull_bar[buf], (uint32_t)((k >> 1) & 1));
                if (__any_sync(0xffffffffu, !okw || *abort_v)) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t tcol = tmem + 256u * buf + ((uint32_t)(32 * sp) << 16) + (uint32_t)(32 * g);
                float V[15];
                {
                    float w[15];
                    if (LAYOUT == TC_EXACT2) {
                        ld_window(tcol + 0, hw, w);
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] = 65536.f * w[j];
                        ld_window(tcol + 64, hw, w);
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] = fmaf(256.f, w[j], V[j]);
                        ld_window(tcol + 128, hw, w);
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] = fmaf(256.f, w[j], V[j]);
                        ld_window(tcol + 192, hw, w);
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] += w[j];
                        // column j of the window is (model J TC_MB + 10 g + 5 hw + j / 3, axis j % 3)
                        const float cs = (lane < 15) ? __ldg(scales + (J * TC_MB + 10 * g + 5 * hw) * 3 + lane) : 1.f;
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] *= srow0 * __shfl_sync(0xffffffffu, cs, j);
                    } else if (LAYOUT == TC_BF16X3) {
                        ld_window(tcol + 0, hw, V);
                        ld_window(tcol + 64, hw, w);
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] += w[j];
                        ld_window(tcol + 128, hw, w);
#pragma unroll
                        for (int j = 0; j < 15; ++j) V[j] += w[j];
                    } else {
                        ld_window(tcol + 0, hw, V);
                    }
                }
                // the accumulator buffer is read: hand it back to the MMA warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty_bar[buf]);
                // rounds 0 and 1 of the window in the two halves of the paired FP32 instructions
                float bx[9], by[9];
                assemble_window<0>(V, alpha, mloc, bx);
                assemble_window<1>(V, alpha, mloc, by);
                float2 Hm[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) Hm[e] = make_float2(bx[e], by[e]);
                float2 ev;
                const float2 cv = crmsd_fast_fp32x2(Hm, make_float2(Ga, Ga), make_float2(Gb[0], Gb[1]), invL, &ev);
                emit_pair(cv.x, ev.x, pok[0], Ga, Gb[0], rowbase + b0, a, b0);
                emit_pair(cv.y, ev.y, pok[1], Ga, Gb[1], rowbase + b0 + 3, a, b0 + 3);
                continue;
            }
            // lane (mloc, alpha): row = axis alpha of A model a; in round r its pair is (a, b0 + 3 r)
            const int64_t a = I * TC_MA + 10 * sp + mloc;
            const int64_t b0 = J * TC_MB + 10 * g + alpha;
            const bool lane_ok = lane < 30 && a < N && a >= row_begin && a < row_end;
            const int64_t rowbase = a * N - a * (a + 1) / 2 - a - 1 - out_base;  // condensed index - b
            float srow0 = 1.f, Ga = 0.f;
            if (lane_ok) {
                srow0 = scales[a * 3 + alpha];
                Ga = G32[a];
            }
            bool pok[4];
            float Gb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t b = b0 + 3 * r;
                pok[r] = lane_ok && (3 * r + alpha) < 10 && b < N && a < b;
                Gb[r] = pok[r] ? __ldg(G32 + b) : 0.f;
            }
            const int buf = (int)(k & 1);
            const bool okw = mbar_wait_sleep(&tfull_bar[buf], (uint32_t)((k >> 1) & 1));
            if (__any_sync(0xffffffffu, !okw || *abort_v)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            tc_fence_after();
            const uint32_t trow = tmem + 256u * buf + ((uint32_t)(32 * sp) << 16) + (uint32_t)(32 * g);
            float V[32];
            {
                float tt[32];
                if (LAYOUT == TC_EXACT2) {
                    // two classes per wait: hh and hl, then lh and ll
                    uint32_t u0[32], u1[32];
                    tmem_ld32_issue(trow + 0, u0);
                    tmem_ld32_issue(trow + 64, u1);
                    tmem_wait_ld();
                    tmem_pin32(u0);
                    tmem_pin32(u1);
#pragma unroll
                    for (int j = 0; j < 32; ++j) V[j] = fmaf(256.f, __uint_as_float(u1[j]), 65536.f * __uint_as_float(u0[j]));
                    tmem_ld32_issue(trow + 128, u0);
                    tmem_ld32_issue(trow + 192, u1);
                    tmem_wait_ld();
                    tmem_pin32(u0);
                    tmem_pin32(u1);
#pragma unroll
                    for (int j = 0; j < 32; ++j) V[j] = fmaf(256.f, __uint_as_float(u0[j]), V[j]) + __uint_as_float(u1[j]);
                    // column j of this warp's 32 is (model b_base + 10 g + j / 3, axis j % 3)
                    const float cs = (lane < 30) ? __ldg(scales + (J * TC_MB + 10 * g) * 3 + lane) : 1.f;
#pragma unroll
                    for (int j = 0; j < 30; ++j) V[j] *= srow0 * __shfl_sync(0xffffffffu, cs, j);
                } else if (LAYOUT == TC_BF16X3) {
                    tmem_ld32(trow + 0, V);
                    tmem_ld32(trow + 64, tt);
#pragma unroll
                    for (int j = 0; j < 32; ++j) V[j] += tt[j];
                    tmem_ld32(trow + 128, tt);
#pragma unroll
                    for (int j = 0; j < 32; ++j) V[j] += tt[j];
                } else {
                    tmem_ld32(trow + 0, V);
                }
            }
            // the accumulator buffer is read: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty_bar[buf]);
            auto emit = [&](float cv, float ev, bool pk, float gbh, int64_t b) {
                emit_pair(cv, ev, pk, Ga, gbh, rowbase + b, a, b);
            };
            if constexpr (!ROT) {
                // two rounds at a time (rounds 2 d and 2 d + 1 in the two halves of the paired FP32
                // instructions): two independent pairs per lane, half the instructions per pair
#pragma unroll 1
                for (int d = 0; d < 2; ++d) {
                    float bx[9], by[9];
                    if (d == 0) {  // warp-uniform; compile-time column offsets in each branch
                        assemble_block(V, 0, alpha, mloc, bx);
                        assemble_block(V, 1, alpha, mloc, by);
                    } else {
                        assemble_block(V, 2, alpha, mloc, bx);
                        assemble_block(V, 3, alpha, mloc, by);
                    }
                    float2 Hm[9];
#pragma unroll
                    for (int e = 0; e < 9; ++e) Hm[e] = make_float2(bx[e], by[e]);
                    float2 ev;
                    const float2 cv = crmsd_fast_fp32x2(Hm, make_float2(Ga, Ga), make_float2(Gb[0], Gb[1]), invL, &ev);
                    emit(cv.x, ev.x, pok[0], Gb[0], b0 + 6 * d);
                    emit(cv.y, ev.y, pok[1], Gb[1], b0 + 6 * d + 3);
                    Gb[0] = Gb[2];
                    Gb[1] = Gb[3];
                    pok[0] = pok[2];
                    pok[1] = pok[3];
                }
            } else {
                // with rotations: one round at a time (a compact loop: the fast path's code size, not
                // its latency, limits this kernel)
#pragma unroll 1
                for (int r = 0; r < 4; ++r) {
                    float blk[9];
                    switch (r) {  // warp-uniform; compile-time column offsets in each case
                        case 0: assemble_block(V, 0, alpha, mloc, blk); break;
                        case 1: assemble_block(V, 1, alpha, mloc, blk); break;
                        case 2: assemble_block(V, 2, alpha, mloc, blk); break;
                        default: assemble_block(V, 3, alpha, mloc, blk); break;
                    }
                    float sv, ev;
                    float m[9], R[9];
                    bool okR = false;
                    const float cv = ROT ? crmsd_fast_rot_fp32(blk, Ga, Gb[0], invL, &sv, &ev, m, R, &okR)
                                         : crmsd_fast_fp32(blk, Ga, Gb[0], invL, &sv, &ev);
                    const int64_t b = b0 + 3 * r;
                    if (ROT) {
                        if (pok[0]) {
                            // blk's rows are axes alpha, alpha + 1, alpha + 2: axis ax is row (ax - alpha) mod 3
                            const int64_t ridx = rowbase + b;
                            bool done = okR;
                            if (!okR) {
                                const unsigned long long slot = atomicAdd(fix_count, 1ull);
                                if ((int64_t)slot < fix_cap) {
                                    RotFix *f = fix + slot;
                                    f->idx = ridx;
#pragma unroll
                                    for (int ax = 0; ax < 3; ++ax) {
                                        const int src = (ax + 3 - alpha) % 3;
#pragma unroll
                                        for (int be = 0; be < 3; ++be)
                                            f->m[3 * ax + be] = sel3(src, m[be], m[3 + be], m[6 + be]);
                                    }
                                } else {
                                    rotation_robust(m, R);  // the list is full: solve it here
                                    done = true;
                                }
                            }
                            if (done) {
                                float Rn[9];
#pragma unroll
                                for (int ax = 0; ax < 3; ++ax) {
                                    const int src = (ax + 3 - alpha) % 3;
#pragma unroll
                                    for (int be = 0; be < 3; ++be) Rn[3 * ax + be] = sel3(src, R[be], R[3 + be], R[6 + be]);
                                }
                                store_rot(rot + ridx * ROT_STRIDE, Rn);
                            }
                        }
                    }
                    emit(cv, ev, pok[0], Gb[0], b);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        Gb[i] = Gb[i + 1];
                        pok[i] = pok[i + 1];
                    }
                }
            }
        }
        if (SPARSE && fill > 0) publish(fill);
        if (LAYOUT == TC_EXACT2 && lane == 0) fl_cnt[blockIdx.x * fw_epi(WIN) + ew] = (unsigned)nfl;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (lane == 0 && *abort_v) {
            // a stopped CTA: the copies of the last FW_STAGES armed stages may still be in flight
            // (the MMA issuer stopped waiting for them); they land before the CTA leaves (bounded)
            for (int64_t r = (q > FW_STAGES ? q - FW_STAGES : 0); r < q; ++r)
                mbar_wait(&full_bar[r % FW_STAGES], (uint32_t)((r / FW_STAGES) & 1));
        }
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
}

// ---- host side ----------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

inline int tc_supported(int form, int64_t L)
{
    if (form == CLUSCO_FORM_BF16_EXACT2 && L > 1024) return CLUSCO_EUNSUPPORTED;  // exact class sums need L <= 1024
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CLUSCO_ECUDA;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return CLUSCO_EUNSUPPORTED;  // built for sm_103a only
    if (!encode_fn()) return CLUSCO_EUNSUPPORTED;
    return CLUSCO_OK;
}

inline int make_map(CUtensorMap *m, void *base, bool tf32, int64_t Lp, int64_t rows, uint32_t box_rows,
                    std::string &err)
{
    const cuuint64_t dims[2] = {(cuuint64_t)Lp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(Lp * (tf32 ? 4 : 2))};
    const cuuint32_t box[2] = {tf32 ? 32u : 64u, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base,
                             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

// Row a of condensed index idx (the largest a with condensed_idx(a, a + 1, N) <= idx). The
// start counts from the nearer end of the triangle, where the quadratic's root is well
// conditioned: from the top, a = (t - sqrt(t^2 - 8 idx)) / 2 with t = 2N - 1; from the bottom,
// the r = N - 1 - a last rows hold r (r + 1) / 2 pairs, so r = ceil((sqrt(8 R + 1) - 1) / 2)
// for the R = P - idx pairs from idx on. In FP32 (N <= 2^22) either start is within a row;
// exact integer corrections follow.
__device__ __forceinline__ int64_t condensed_row(int64_t idx, int64_t N)
{
    const int64_t P = N * (N - 1) / 2;
    int64_t a;
    if (N <= ((int64_t)1 << 22)) {
        if (2 * idx < P) {
            const float t = 2.f * (float)N - 1.f;
            a = (int64_t)floorf(0.5f * (t - sqrtf(fmaxf(t * t - 8.f * (float)idx, 0.f))));
        } else {
            const float R = (float)(P - idx);
            a = N - 1 - (int64_t)ceilf(0.5f * (sqrtf(8.f * R + 1.f) - 1.f));
        }
    } else {
        const double t = 2.0 * (double)N - 1.0;
        a = (int64_t)floor(0.5 * (t - sqrt(fmax(t * t - 8.0 * (double)idx, 0.0))));
    }
    a = a < 0 ? 0 : (a > N - 2 ? N - 2 : a);
    while (a > 0 && condensed_idx(a, a + 1, N) > idx) --a;
    while (a < N - 2 && condensed_idx(a + 1, a + 2, N) <= idx) ++a;
    return a;
}

// 4-way signed byte dot product with a 32-bit accumulator.
__device__ __forceinline__ int dp4a_ss(int a, int b, int c)
{
    int d;
    asm("dp4a.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// The flagged-pair lists of the exact-digit forward: one per epilogue warp (slot CTA x epilogue
// warps per CTA + warp), FL_MAXSLOTS slots at most, each of capacity flist_entries / slots;
// their counts follow the flag mask (flag_list_offset words from its start, 16-byte aligned).
constexpr int FL_MAXSLOTS = 4096;
inline int64_t flag_list_offset(int64_t npairs) { return ((npairs + 31) / 32 + 3) / 4 * 4; }
// list entries for a pair range: 1/32 of the pairs (the bench ensembles flag under 1 %), at
// least 2^16 and at most 2^27 (1 GiB of workspace; past that, and past a list's share, the
// pairs take the mask path), so that the counts and their prefix sums stay below 2^32
inline int64_t flag_list_entries(int64_t npairs)
{
    return std::min<int64_t>(std::max<int64_t>(npairs / 32, (int64_t)1 << 16), (int64_t)1 << 27);
}

// Minimum flagged pairs per refinement warp: fewer warps with fuller batches where the flagged
// set is small (each batch costs its FP64 instructions whatever its fill).
constexpr int REFINE_MIN_PAIRS = 16;

// The pairs the fast path flagged: each one's covariance recomputed exactly from the 16-bit
// fixed-point coordinates n = 256 h + l (byte planes, h and l signed; rows in the tensor-core
// layout, zero past L) as three digit classes of nine sums, hh, hl + lh and ll, each an exact
// 32-bit integer (signed 4-way byte dot products over atom quads: per atom |hh|, |ll| <= 2^14
// and |hl + lh| <= 2^15, so over L <= 1024 atoms every class stays below 2^25 and each is
// reduced across the warp on its own), then H = 65536 hh + 256 (hl + lh) + ll in int64, scaled
// to FP64, and cRMSD by FP64 Newton from an FP32 start (crmsd_refine_newton_fp64). Lanes split
// the atoms of each pair, and pairs are batched 32 at a time so that every FP64 instruction runs
// on 32 lanes. The flagged pairs come as the forward's per-warp lists (fl_cnt[s] pairs in slot
// s, the ones past fl_cap in the mask): each block scans the list counts; with F listed pairs,
// warp g of the W' = min(W, ceil(F / REFINE_MIN_PAIRS)) working warps (interleaved across the
// blocks, so across the SMs) takes ranks [g F / W', (g + 1) F / W') of the concatenated lists,
// so the work is balanced however the flagged pairs cluster. Pairs past a list's capacity
// (their mask bits) are taken after it, mask words round-robin over all warps.
// Two CTAs per SM (the launch bound keeps the FP64 Newton and a pair's twelve 16-byte loads in
// 128 registers); three would cap them at 80, and the loads would spill.
__global__ void __launch_bounds__(256, 2) refine_flagged_kernel(const int8_t *__restrict__ hplane,
                                                                   const int8_t *__restrict__ lplane,
                                                                   const float *__restrict__ scales,
                                                                   const double *__restrict__ G64, int64_t N, int L,
                                                                   int Lp, int64_t npairs, int64_t out_base,
                                                                   const uint32_t *__restrict__ flags,
                                                                   const int2 *__restrict__ flist,
                                                                   const unsigned *__restrict__ fl_cnt, int nslots,
                                                                   int fl_cap, PairSink sink)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const double invL = 1.0 / (double)L;
    // the warp's batch: slot j holds the j-th pair's models (lst) and its three exact class
    // sums per covariance entry (sv: hh, then hl + lh, then ll); the FP64 work waits for the
    // batch, where every FP64 instruction serves 32 pairs
    __shared__ int2 lst[8][32];
    __shared__ int sv[8][27][32];
    __shared__ unsigned spre[FL_MAXSLOTS + 1];
    int cnt = 0;
    auto flush = [&]() {
        __syncwarp();
        float c = 0.f;
        int64_t oidx = 0;
        if (lane < cnt) {
            const int64_t sa = lst[wib][lane].x, sb = lst[wib][lane].y;
            oidx = condensed_idx(sa, sb, N) - out_base;
            float s3a[3], s3b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                s3a[k] = scales[sa * 3 + k];
                s3b[k] = scales[sb * 3 + k];
            }
            const double Ga = G64[sa], Gb = G64[sb];
            // the FP32 start from the same sums in FP32 (it only has to be close: Newton in FP64
            // polishes it), the exact covariance in FP64 (each scale product is exact in FP64)
            const float nrmf = __fdividef(2.f, (float)(Ga + Gb));
            float mf[9];
            double H[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const long long vk = 65536LL * sv[wib][k][lane] + 256LL * sv[wib][9 + k][lane] + sv[wib][18 + k][lane];
                mf[k] = (float)vk * (s3a[k / 3] * s3b[k % 3]) * nrmf;
                H[k] = (double)vk * ((double)s3a[k / 3] * (double)s3b[k % 3]);
            }
            c = crmsd_refine_newton_fp64(H, Ga, Gb, invL, sigma_hat_f32(mf));
            if (!sink.list) sink.out[oidx] = c;
        }
        if (sink.list) sink_append_warp(sink, lane < cnt && c < sink.tau, oidx + out_base, c);
        __syncwarp();
        cnt = 0;
    };
    // one flagged pair (a < b): its exact class sums reduced across the warp into slot cnt. Each
    // lane takes 16 consecutive bytes (16 atoms) of each of the pair's twelve rows per 512-byte
    // chunk, so a pair of L <= 512 atoms costs one round of twelve 16-byte loads
    auto pair = [&](int64_t a, int64_t b) {
        const int8_t *ha = hplane + tc_row(a, 0) * Lp;
        const int8_t *la = lplane + tc_row(a, 0) * Lp;
        const int8_t *hb = hplane + tc_row(b, 0) * Lp;
        const int8_t *lb = lplane + tc_row(b, 0) * Lp;
        int hh[9], hx[9], ll[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            hh[k] = 0;
            hx[k] = 0;
            ll[k] = 0;
        }
#pragma unroll 1
        for (int o = 16 * lane; o < Lp; o += 512) {
            int A[3][4], Al[3][4], B[3][4], Bl[3][4];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const int4 u = __ldg(reinterpret_cast<const int4 *>(ha + ax * Lp + o));
                const int4 ul = __ldg(reinterpret_cast<const int4 *>(la + ax * Lp + o));
                const int4 w = __ldg(reinterpret_cast<const int4 *>(hb + ax * Lp + o));
                const int4 wl = __ldg(reinterpret_cast<const int4 *>(lb + ax * Lp + o));
                A[ax][0] = u.x, A[ax][1] = u.y, A[ax][2] = u.z, A[ax][3] = u.w;
                Al[ax][0] = ul.x, Al[ax][1] = ul.y, Al[ax][2] = ul.z, Al[ax][3] = ul.w;
                B[ax][0] = w.x, B[ax][1] = w.y, B[ax][2] = w.z, B[ax][3] = w.w;
                Bl[ax][0] = wl.x, Bl[ax][1] = wl.y, Bl[ax][2] = wl.z, Bl[ax][3] = wl.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) {
                        const int k = 3 * al + be;
                        hh[k] = dp4a_ss(A[al][j], B[be][j], hh[k]);
                        hx[k] = dp4a_ss(Al[al][j], B[be][j], dp4a_ss(A[al][j], Bl[be][j], hx[k]));
                        ll[k] = dp4a_ss(Al[al][j], Bl[be][j], ll[k]);
                    }
        }
        const int slot = cnt;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int shh = __reduce_add_sync(0xffffffffu, hh[k]);
            const int shx = __reduce_add_sync(0xffffffffu, hx[k]);
            const int sll = __reduce_add_sync(0xffffffffu, ll[k]);
            if (lane == k) {
                sv[wib][k][slot] = shh;
                sv[wib][9 + k][slot] = shx;
                sv[wib][18 + k][slot] = sll;
            }
        }
        if (lane == 0) lst[wib][slot] = make_int2((int)a, (int)b);
        if (++cnt == 32) flush();
    };

    // the list counts (each capped at fl_cap) and their exclusive prefix sums, per block
    bool over = false;
    {
        const int per = (nslots + 255) / 256;
        const int i0 = min((int)threadIdx.x * per, nslots), i1 = min(i0 + per, nslots);
        unsigned loc = 0;
        for (int i = i0; i < i1; ++i) {
            const unsigned c = fl_cnt[i];
            over |= c > (unsigned)fl_cap;
            loc += min(c, (unsigned)fl_cap);
        }
        unsigned inc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        __shared__ unsigned wtot[8];
        if (lane == 31) wtot[wib] = inc;
        __syncthreads();
        unsigned run = inc - loc;
        for (int w = 0; w < wib; ++w) run += wtot[w];
        for (int i = i0; i < i1; ++i) {
            spre[i] = run;
            run += min(fl_cnt[i], (unsigned)fl_cap);
        }
        if (threadIdx.x == 255) spre[nslots] = run;
        over = __syncthreads_or(over);
    }
    const unsigned F = spre[nslots];
    const unsigned W = gridDim.x * (blockDim.x >> 5);
    const unsigned Wf = max(1u, min(W, (F + REFINE_MIN_PAIRS - 1) / REFINE_MIN_PAIRS));
    const unsigned g = wib * gridDim.x + blockIdx.x;
    if (g < Wf) {
        const unsigned r0 = (unsigned)((unsigned long long)g * F / Wf);
        const unsigned r1 = (unsigned)((unsigned long long)(g + 1) * F / Wf);
        for (unsigned r = r0; r < r1; r += 32) {
            // lane j fetches the pair of rank r + j: its slot by bisection of the prefix sums
            const unsigned rr = r + lane;
            int2 e = make_int2(0, 0);
            if (rr < r1) {
                int lo = 0, hi = nslots;  // spre[lo] <= rr < spre[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (spre[mid] <= rr)
                        lo = mid;
                    else
                        hi = mid;
                }
                e = flist[(int64_t)lo * fl_cap + (rr - spre[lo])];
            }
            const int n = (int)min(32u, r1 - r);
            for (int j = 0; j < n; ++j) pair(__shfl_sync(0xffffffffu, e.x, j), __shfl_sync(0xffffffffu, e.y, j));
        }
        if (cnt) flush();
    }
    if (!over) return;
    // pairs past a list's capacity: their mask bits, words w0 + W (32 it + j), lane j loading one
    // word per iteration (32 loads at a time)
    const int64_t nwords = (npairs + 31) / 32;
    for (int64_t base = g; base < nwords; base += 32 * (int64_t)W) {
        const int64_t wl = base + (int64_t)lane * W;
        uint32_t word = wl < nwords ? flags[wl] : 0u;
        if (wl == nwords - 1 && (npairs & 31)) word &= ~0u >> (32 - (int)(npairs & 31));
        uint32_t nz = __ballot_sync(0xffffffffu, word != 0u);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            const int64_t wi = base + (int64_t)src * W;
            uint32_t wd = __shfl_sync(0xffffffffu, word, src);
            while (wd) {
                const int bit = __ffs(wd) - 1;
                wd &= wd - 1;
                const int64_t idx = wi * 32 + bit + out_base;
                const int64_t a = condensed_row(idx, N);
                pair(a, idx - condensed_idx(a, a + 1, N) + a + 1);
            }
        }
    }
    if (cnt) flush();
}

template <int LAYOUT>
inline int launch_tc(const TcArgs &a, cudaStream_t st, std::string &err)
{
    const bool tf32 = LAYOUT == TC_TF32;
    const int64_t rows = tf32 ? a.Rpad : 2 * a.Rpad;
    CUtensorMap mA, mB;
    int rc;
    if ((rc = make_map(&mA, a.planes, tf32, a.Lp, rows, 128, err))) return rc;
    if ((rc = make_map(&mB, a.planes, tf32, a.Lp, rows, 64, err))) return rc;
    const int64_t Npad = a.Rpad / 32 * 10;
    const int64_t TA = Npad / TC_MA, TB = Npad / TC_MB;
    const int64_t I0 = a.row_begin / TC_MA, I1 = (a.row_end - 1) / TC_MA + 1;
    const int64_t t0 = tc_row_start(I0, TB), nt = tc_row_start(I1, TB) - t0;
    const int nkb = (int)(a.Lp / (tf32 ? 32 : 64));
    if (nt <= 0) return CLUSCO_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool win = !a.rot && a.Lp <= FW_WIN_MAXLP;
    auto kern = a.rot ? pairs_tc_kernel<LAYOUT, true, false>
                      : (a.list ? (win ? pairs_tc_kernel<LAYOUT, false, true, true> : pairs_tc_kernel<LAYOUT, false, true>)
                                : (win ? pairs_tc_kernel<LAYOUT, false, false, true> : pairs_tc_kernel<LAYOUT, false, false>));
    PairSink sink;
    sink.out = a.out;
    sink.out_base = a.out_base;
    sink.list = a.list;
    sink.vals = a.vals;
    sink.count = a.count;
    sink.cap = a.cap;
    sink.tau = a.tau;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FW_SMEM);
    if (e != cudaSuccess) {
        err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    // persistent: one CTA per SM, CTA x takes tiles x, x + grid, x + 2 grid, ...
    const unsigned grid = (unsigned)std::min<int64_t>(nt, sms > 0 ? sms : 148);
    const int64_t npairs = condensed_idx(a.row_end - 1, a.N - 1, a.N) + 1 - a.out_base;
    const int64_t nslots = (int64_t)grid * fw_epi(win);  // one flagged-pair list per epilogue warp
    if (nslots > FL_MAXSLOTS) {
        err = "more epilogue warps than flagged-pair list slots";
        return CLUSCO_EUNSUPPORTED;
    }
    int fl_cap = a.flist ? (int)std::min<int64_t>(a.flist_entries / nslots, 1 << 30) : 0;
#ifdef CLUSCO_DEBUG_HOOKS
    if (debug_fl_cap() > 0) fl_cap = std::min(fl_cap, debug_fl_cap());
#endif
    if (LAYOUT == TC_EXACT2) {
        // the mask and the list counts
        e = cudaMemsetAsync(a.flags, 0, (size_t)(flag_list_offset(npairs) + FL_MAXSLOTS) * sizeof(uint32_t), st);
        if (e != cudaSuccess) {
            err = std::string("flag mask reset: ") + cudaGetErrorString(e);
            return CLUSCO_ECUDA;
        }
    }
    if (a.list) {
        e = cudaMemsetAsync(a.count, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) {
            err = std::string("list count reset: ") + cudaGetErrorString(e);
            return CLUSCO_ECUDA;
        }
    }
    prof_mark(PROF_PAIRS, st);
    if (a.rot) {
        e = cudaMemsetAsync(a.fix_count, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) {
            err = std::string("rotation list reset: ") + cudaGetErrorString(e);
            return CLUSCO_ECUDA;
        }
    }
    kern<<<grid, fw_threads(win), FW_SMEM, st>>>(mA, mB, a.scales, a.G32, a.N, (int)a.L, nkb, a.Rpad, TA, TB, t0, nt,
                                             a.row_begin, a.row_end, sink, a.rot, a.fix, a.fix_count, a.fix_cap,
                                             a.flags, a.flist, a.flags ? a.flags + flag_list_offset(npairs) : nullptr,
                                             fl_cap);
    e = cudaGetLastError();
    prof_mark(PROF_PAIRS, st);
    if (e == cudaSuccess && LAYOUT == TC_EXACT2) {
        // one wave of two CTAs per SM
        const int nsm = sms > 0 ? sms : 148;
        refine_flagged_kernel<<<2 * nsm, 256, 0, st>>>(a.hplane, a.lplane, a.scales, a.G64, a.N, (int)a.L,
                                                        (int)a.Lp, npairs, a.out_base, a.flags, a.flist,
                                                        a.flags + flag_list_offset(npairs), (int)nslots,
                                                        fl_cap, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && a.rot) {
        rot_fixup_kernel<<<4 * (sms > 0 ? sms : 148), 256, 0, st>>>(a.fix, a.fix_count, a.fix_cap, a.rot);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("pairs_tc_kernel launch: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

inline int tc_launch_allpairs(const TcArgs &a, cudaStream_t st, std::string &err)
{
    if (a.form == CLUSCO_FORM_BF16_EXACT2) return launch_tc<TC_EXACT2>(a, st, err);
    if (a.form == CLUSCO_FORM_BF16X3) return launch_tc<TC_BF16X3>(a, st, err);
    return launch_tc<TC_TF32>(a, st, err);
}

}  // namespace clusco

// bwd_tc.cuh -- adjoint of the all-pairs matrix on the tensor cores (tcgen05).
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// One CTA owns one A tile I (40 models = 128 rows of the operand planes) and a contiguous
// range of B tiles J over the full square (every b != a in both orders, so the CTA owns its
// rows and needs no atomics). Tensor memory (512 columns) holds
//   cols [0, 192)        the tile covariance in three exact digit classes (hh, hl + lh, ll);
//   cols [192, 192 + Lp) the CTA's sum P.X over its column range (128 rows x Lp atoms,
//                        FP32), accumulated over the whole sweep.
// Three roles run as a pipeline over the tiles J, synchronised by mbarriers:
//   warp 0 (TMA): streams the covariance operands (2-stage ring, 128-byte swizzle) and, one
//     tile behind, the transposed TF32 hi / lo coordinates X_J^T in 64-atom chunks (double
//     buffer);
//   warp 1 (MMA): GEMM1 = exact-digit covariance of tile J (tcgen05 kind::f16, hl and lh summed
//     in one class: |hl + lh| <= 2^15 per atom keeps the sum exact for L <= 512), then
//     GEMM2 of tile J-1 = sum += P . X (tcgen05 kind::tf32, three passes hi.hi + hi.lo + lo.hi,
//     about 2^-21 relative per product);
//   warps 2-9 (epilogue): read tile J's covariance from TMEM (then release it to GEMM1 of
//     J+1), assemble each 3x3 block (rows cyclic, as in the forward), take Sigma from the
//     FP32 fast path and the rotation with it (dSigma/dM from the quartic; Horn's adjugate,
//     or Jacobi sweeps, only near a double root), undo the cyclic order and write w~ R as two
//     TF32 parts into a shared 128 x 64 operand in the 128-byte-swizzled K-major layout;
//     pairs below the near-duplicate threshold go to the FP64 direct kernel.
// So tile J's rotations overlap GEMM1 of J+1 and GEMM2 of J-1. Rotations live only in shared
// memory. At the end the epilogue reads the sum out of TMEM into the CTA's partial-gradient
// slice (negated); bwd_reduce_kernel adds the partials of the S column ranges, the diagonal
// term and the centring projection. Requires Lp = ceil(L/64)*64 <= 320.
#pragma once
#include "backward.cuh"
#include "pairs_tc.cuh"
#include "rotation.cuh"

namespace clusco {

constexpr int BT_STAGES = 2;
constexpr int BT_THREADS = 320;                           // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int BT_MAXLP = 320;
constexpr uint32_t BT_TMEM_COLS = 512;
constexpr uint32_t BT_D2 = 192;                            // first TMEM column of the P.X sum
constexpr size_t BT_RING = BT_STAGES * STAGE_BYTES_BF16;   // 96 KB; reused for X_J^T chunks
constexpr size_t BT_A2 = 2 * 128 * 64 * 4;                 // hi, lo: 64 KB
constexpr int BT_XCH = 64;                                 // atoms per X^T chunk (GEMM2 N)
constexpr size_t BT_XBUF = 4 * BT_XCH * 128;               // hi/lo x two 32-column blocks: 32 KB
constexpr size_t BT_XT = 2 * BT_XBUF;                      // double buffer
constexpr size_t BT_SMEM = 1024 + BT_RING + BT_XT + BT_A2;

struct BtWs {
    void *planes = nullptr;  // EXACT2 digit planes [2][Rpad][Lp] bf16
    float *scales = nullptr;
    double *G64 = nullptr;
    float *G32 = nullptr;
    float *xf = nullptr;     // [Rpad][Lp] centred FP32, padded row layout
    float *xT = nullptr;     // [2][Lp][Rpad] TF32 hi / lo parts, transposed
    float *Gp = nullptr;     // [S][Rpad][Lp] partial gradients
    float *dp = nullptr;     // [S][Npad] partial row sums of w~
    long long *nd_list = nullptr;
    unsigned long long *nd_count = nullptr;
    unsigned *scl = nullptr;  // stored-rotation adjoint: max |centred x|, max |w| (float bits)
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
    w.xT = (float *)take(sizeof(float) * 2 * w.Lp * w.Rpad);
    w.Gp = (float *)take(sizeof(float) * w.S * w.Rpad * w.Lp);
    w.dp = (float *)take(sizeof(float) * w.S * w.Npad);
    const int64_t P = N * (N - 1) / 2;
    w.nd_cap = P < (int64_t)(1 << 22) ? P : (int64_t)(1 << 22);
    w.nd_list = (long long *)take(sizeof(long long) * 2 * w.nd_cap);
    w.nd_count = (unsigned long long *)take(sizeof(unsigned long long));
    w.scl = (unsigned *)take(2 * sizeof(unsigned));
    w.bytes = off;
    return w;
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    return __uint_as_float(t);
}

// Byte offset of element (row r, column c) of a 128 x 64 FP32 K-major operand stored as two
// 128-byte-swizzled column blocks of 32 elements (16 KB each): the 16-byte chunk index of
// a row is XORed with the row index mod 8, as the TMA writes and tcgen05.mma reads it.
__device__ __forceinline__ uint32_t a2_offset(int r, int c)
{
    const int kb2 = c >> 5, e = c & 31;
    return (uint32_t)(kb2 * 16384 + r * 128 + ((((e >> 2) ^ (r & 7)) & 7) << 4) + ((e & 3) << 2));
}

// xT[s][i][r] = TF32 part s of xf[r][i]; 32 x 32 tiles through shared memory.
__global__ void __launch_bounds__(256) bt_transpose_kernel(const float *__restrict__ xf, int64_t Rpad, int Lp,
                                                           float *__restrict__ xT)
{
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) t[k][tx] = xf[(r0 + k) * Lp + i0 + tx];
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const float v = t[tx][k];
        const float hi = tf32_rna(v);
        xT[(int64_t)(i0 + k) * Rpad + r0 + tx] = hi;
        xT[((int64_t)Lp + i0 + k) * Rpad + r0 + tx] = tf32_rna(v - hi);
    }
}

__global__ void __launch_bounds__(BT_THREADS, 1)
    bwd_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapX, const float *__restrict__ scales,
                  const float *__restrict__ G32, int64_t N, int L, int Lp, int nkb, int64_t Rpad, int64_t TB, int64_t S,
                  int64_t JC, const float *__restrict__ crmsd, const float *__restrict__ wvec, float eps,
                  float *__restrict__ Gp, float *__restrict__ dp, long long *__restrict__ nd_list,
                  unsigned long long *__restrict__ nd_count, int64_t nd_cap)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[BT_STAGES];   // GEMM1 ring: K block landed
    __shared__ __align__(8) uint64_t empty_bar[BT_STAGES];  // GEMM1 ring: K block consumed
    __shared__ __align__(8) uint64_t done1_bar;             // GEMM1 of a tile is in TMEM
    __shared__ __align__(8) uint64_t tfree_bar;             // the epilogue has read that tile (8 arrivals)
    __shared__ __align__(8) uint64_t a2full_bar;            // the rotation operand is written (8 arrivals)
    __shared__ __align__(8) uint64_t a2empty_bar;           // GEMM2 has finished reading it
    __shared__ __align__(8) uint64_t xfull_bar[2];          // an X^T chunk landed in buffer 0 / 1
    __shared__ __align__(8) uint64_t xempty_bar[2];         // GEMM2 has finished reading buffer 0 / 1
    __shared__ __align__(8) uint64_t d2_bar;                // the last GEMM2 has finished
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float sB_scale[TC_MB * 3];
    __shared__ float sB_G32[TC_MB];
    __shared__ float dsum[TC_MA];

    // 1024-byte aligned in the shared window; indexing smem_raw (not an integer cast) keeps the
    // pointer in the shared address space, so accesses through it compile to shared loads/stores
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase0 = smem_u32(smem);
    uint8_t *XT = smem + BT_RING;            // two X^T chunk buffers of BT_XBUF bytes
    uint8_t *A2 = smem + BT_RING + BT_XT;    // [hi 32 KB][lo 32 KB]
    const uint32_t xtbase = smem_u32(XT), a2base = smem_u32(A2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t I = blockIdx.x / S, sidx = blockIdx.x % S;
    const int64_t J0 = sidx * JC, J1 = (J0 + JC < TB) ? J0 + JC : TB;
    const int64_t a_base = I * TC_MA;
    const int64_t Npad = Rpad / 32 * 10;

    if (J0 >= J1) {  // an empty column range still owns its (zero) partial slice
        float *gp = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
        for (int e = tid; e < 128 * Lp; e += BT_THREADS) gp[e] = 0.f;
        if (tid < TC_MA) dp[sidx * Npad + a_base + tid] = 0.f;
        return;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, BT_TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < BT_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&xfull_bar[s], 1);
            mbar_init(&xempty_bar[s], 1);
        }
        mbar_init(&done1_bar, 1);
        mbar_init(&tfree_bar, 8);
        mbar_init(&a2full_bar, 8);
        mbar_init(&a2empty_bar, 1);
        mbar_init(&d2_bar, 1);
        abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    for (int e = tid; e < (int)(BT_A2 / 16); e += BT_THREADS)
        reinterpret_cast<float4 *>(A2)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < TC_MA) dsum[tid] = 0.f;
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int64_t nJ = J1 - J0;
    const int nch = Lp / BT_XCH;
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        // ================= TMA producer =================
        if (lane == 0) {
            int64_t q = 0, c = 0;
            bool ok = true;
            auto g1_loads = [&](int64_t J) {
                for (int kb = 0; kb < nkb && ok; ++kb, ++q) {
                    const int s = (int)(q % BT_STAGES);
                    const int64_t use = q / BT_STAGES;
                    if (q >= BT_STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                        ok = false;
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
            };
            auto xt_loads = [&](int64_t J) {
                for (int ch = 0; ch < nch && ok; ++ch, ++c) {
                    const int buf = (int)(c & 1);
                    const int64_t use = c >> 1;
                    if (c >= 2 && !mbar_wait(&xempty_bar[buf], (uint32_t)((use - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&xfull_bar[buf], (uint32_t)BT_XBUF);
#pragma unroll
                    for (int sp2 = 0; sp2 < 2; ++sp2)
#pragma unroll
                        for (int kb2 = 0; kb2 < 2; ++kb2)
                            tma_load_2d(XT + buf * BT_XBUF + (2 * sp2 + kb2) * (BT_XCH * 128), &mapX,
                                        &xfull_bar[buf], (int)(64 * J + 32 * kb2), (int)(sp2 * Lp + ch * BT_XCH));
                }
            };
            for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) {
                g1_loads(J0 + j);
                if (j >= 1) xt_loads(J0 + j - 1);
            }
            if (ok && !*abort_v) xt_loads(J1 - 1);
            if (!ok) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            int64_t q = 0, c = 0;
            bool ok = true;
            constexpr uint32_t id64 = make_idesc(128, 64, 1);
            constexpr uint32_t idx = make_idesc(128, BT_XCH, 2);
            auto g1 = [&]() {
                for (int kb = 0; kb < nkb && ok; ++kb, ++q) {
                    const int s = (int)(q % BT_STAGES);
                    const int64_t use = q / BT_STAGES;
                    if (!mbar_wait(&full_bar[s], (uint32_t)(use & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = sbase0 + s * STAGE_BYTES_BF16;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        const uint64_t ah = desc_sw128(sb + 32 * k), al = desc_sw128(sb + 16384 + 32 * k);
                        const uint64_t bh = desc_sw128(sb + 32768 + 32 * k), bl = desc_sw128(sb + 40960 + 32 * k);
                        mma_bf16(tmem + 0, ah, bh, id64, acc);
                        mma_bf16(tmem + 64, ah, bl, id64, acc);
                        mma_bf16(tmem + 64, al, bh, id64, 1u);
                        mma_bf16(tmem + 128, al, bl, id64, acc);
                    }
                    mma_commit(&empty_bar[s]);
                }
                mma_commit(&done1_bar);
            };
            auto g2 = [&](int64_t jj) {
                if (!mbar_wait(&a2full_bar, (uint32_t)(jj & 1))) {
                    ok = false;
                    return;
                }
                tc_fence_after();
                for (int ch = 0; ch < nch && ok; ++ch, ++c) {
                    const int buf = (int)(c & 1);
                    if (!mbar_wait(&xfull_bar[buf], (uint32_t)((c >> 1) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xb = xtbase + buf * BT_XBUF;
                    const uint32_t d = tmem + BT_D2 + (uint32_t)(ch * BT_XCH);
#pragma unroll
                    for (int kb2 = 0; kb2 < 2; ++kb2)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t ahi = desc_sw128(a2base + kb2 * 16384 + 32 * k);
                            const uint64_t alo = desc_sw128(a2base + 32768 + kb2 * 16384 + 32 * k);
                            const uint64_t bhi = desc_sw128(xb + kb2 * (BT_XCH * 128) + 32 * k);
                            const uint64_t blo = desc_sw128(xb + (2 + kb2) * (BT_XCH * 128) + 32 * k);
                            // each chunk's first MMA of the sweep starts its columns from zero
                            mma_tf32(d, ahi, bhi, idx, (jj == 0 && kb2 == 0 && k == 0) ? 0u : 1u);
                            mma_tf32(d, ahi, blo, idx, 1u);
                            mma_tf32(d, alo, bhi, idx, 1u);
                        }
                    mma_commit(&xempty_bar[buf]);
                }
                mma_commit(&a2empty_bar);
            };
            for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) {
                if (j >= 1 && !mbar_wait_sleep(&tfree_bar, (uint32_t)((j - 1) & 1))) {
                    ok = false;
                    break;
                }
                g1();
                if (j >= 1 && ok) g2(j - 1);
            }
            if (ok && !*abort_v) g2(nJ - 1);
            mma_commit(&d2_bar);
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
        float srow0 = 1.f, Ga = 0.f;
        if (lane_ok) {
            srow0 = scales[a * 3 + alpha];
            Ga = G32[a];
        }
        const uint32_t trow = tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)(32 * g);
        bool alive = true;
        for (int64_t j = 0; j < nJ; ++j) {
            const int64_t J = J0 + j;
            const int64_t b_base = J * TC_MB;
            if (etid < TC_MB * 3) sB_scale[etid] = scales[(b_base + etid / 3) * 3 + etid % 3];
            if (etid < TC_MB) sB_G32[etid] = G32[b_base + etid];
            // forward outputs and weights of this lane's four pairs (issued early)
            float cpre[4], wpre[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                cpre[r] = 0.f;
                wpre[r] = 0.f;
                const int bq = 3 * r + alpha;
                const int64_t b = b_base + 10 * g + bq;
                if (lane_ok && bq < 10 && b < N && b != a) {
                    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
                    const int64_t idx = condensed_idx(lo, hi, N);
                    cpre[r] = crmsd[idx];
                    wpre[r] = wvec[idx];
                }
            }
            const bool ok1 = mbar_wait_sleep(&done1_bar, (uint32_t)(j & 1));
            if (named_bar_or(1, 256, !ok1 || *abort_v)) {  // uniform across the epilogue warps
                alive = false;
                break;
            }
            tc_fence_after();
            float V[32];
            {
                float t[32];
                tmem_ld32(trow + 0, V);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) V[jj] *= 65536.f;
                tmem_ld32(trow + 64, t);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) V[jj] = fmaf(256.f, t[jj], V[jj]);
                tmem_ld32(trow + 128, t);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) V[jj] += t[jj];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tfree_bar);  // TMEM cols 0..191 may be overwritten now
#pragma unroll
            for (int jj = 0; jj < 30; ++jj) V[jj] *= srow0 * sB_scale[30 * g + jj];
            float Pall[4][9];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float cand[3][3];
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) {
                        const int jj = 9 * r + 3 * al + be;
                        cand[al][be] = (jj < 32) ? V[jj] : 0.f;
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
#pragma unroll
                for (int e = 0; e < 9; ++e) Pall[r][e] = 0.f;
                const int bq = 3 * r + alpha;
                const int lb = 10 * g + bq;
                const int64_t b = b_base + lb;
                if (lane_ok && bq < 10 && b < N && b != a) {
                    const float c = cpre[r], w = wpre[r];
                    if (!(c >= CLUSCO_NEARDUP)) {
                        if (a < b && w != 0.f) {
                            const unsigned long long slot = atomicAdd(nd_count, 1ull);
                            if ((int64_t)slot < nd_cap) {
                                nd_list[2 * slot] = a;
                                nd_list[2 * slot + 1] = b;
                            }
                        }
                    } else if (w != 0.f) {
                        const float nrm = __fdividef(2.f, Ga + sB_G32[lb]);
                        float Hn[9], Rp[9];
#pragma unroll
                        for (int e = 0; e < 9; ++e) Hn[e] = blk[e] * nrm;
                        if (!sigma_rotation_f32(Hn, Rp)) rotation_robust_ptr(Hn, Rp);
                        const float coef = __fdividef(w, (float)L * fmaxf(c, eps));
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const int src_row = (i + 3 - alpha) % 3;
#pragma unroll
                            for (int be = 0; be < 3; ++be)
                                Pall[r][3 * i + be] = coef * sel3(src_row, Rp[be], Rp[3 + be], Rp[6 + be]);
                        }
                        atomicAdd(&dsum[la], coef);
                    }
                }
            }
            // the operand is single-buffered: wait until GEMM2 of the previous tile has read it
            bool ok2 = true;
            if (j >= 1) ok2 = mbar_wait_sleep(&a2empty_bar, (uint32_t)((j - 1) & 1));
            if (named_bar_or(1, 256, !ok2 || *abort_v)) {
                alive = false;
                break;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int bq = 3 * r + alpha;
                if (lane < 30 && bq < 10) {
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            const uint32_t off = a2_offset(32 * sp + 3 * mloc + i, 32 * g + 3 * bq + be);
                            const float v = Pall[r][3 * i + be];
                            const float vh = tf32_rna(v);
                            *reinterpret_cast<float *>(A2 + off) = vh;
                            *reinterpret_cast<float *>(A2 + 32768 + off) = tf32_rna(v - vh);
                        }
                }
            }
            fence_proxy_async();  // generic-proxy stores to A2 must be visible to tcgen05.mma
            __syncwarp();
            if (lane == 0) mbar_arrive(&a2full_bar);
            named_bar_sync(1, 256);  // sB_* of this tile are no longer read
        }
        if (alive) {
            const bool ok3 = mbar_wait_sleep(&d2_bar, 0);
            if (named_bar_or(1, 256, !ok3 || *abort_v)) alive = false;
        }
        if (alive) {
            tc_fence_after();
            // read the P.X sum out of TMEM: warp (sp, g) takes lanes 32 sp.., half of the atoms
            float *row = Gp + (sidx * Rpad + 128 * I + 32 * sp + lane) * (int64_t)Lp;
            const int half = Lp / 2;
            for (int c0 = g * half; c0 < (g + 1) * half; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * sp) << 16) + BT_D2 + (uint32_t)c0, v);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) row[c0 + jj] = -v[jj];
            }
            if (etid < TC_MA) dp[sidx * Npad + a_base + etid] = dsum[etid];
        } else {
            atomicExch(&abort_flag, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_v && tid == 0) {
        // drain (bounded) whatever TMA traffic may still be landing in this CTA's shared memory
        for (int s = 0; s < BT_STAGES; ++s) mbar_wait(&full_bar[s], 0);
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BT_TMEM_COLS);
}

// g_a = sum_s Gp[s] + (sum_s dp[s][a]) x_a, minus its atom mean. One block of three warps per
// model, warp = axis: each lane holds up to four float4 columns of its row (Lp <= 512), every
// partial slice is an independent 16-byte load, the axis mean is a warp reduction, and the
// model's gradient goes out through shared memory as one contiguous [L][3] run. Columns past L
// are zero in every input, so the row sum over Lp is the sum over L.
constexpr int BRED_THREADS = 96;
constexpr int BRED_MAXQ = 4;

__global__ void __launch_bounds__(BRED_THREADS) bwd_reduce_kernel(const float *__restrict__ Gp,
                                                                  const float *__restrict__ dp,
                                                                  const float *__restrict__ xf, int64_t N, int L,
                                                                  int Lp, int64_t Rpad, int64_t S,
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
    for (int64_t s = 0; s < S; ++s) d += dp[s * Npad + a];
    float4 v[BRED_MAXQ];
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < BRED_MAXQ; ++c) {
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
    for (int c = 0; c < BRED_MAXQ; ++c) {
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
    bwd_reduce_kernel<<<(unsigned)N, BRED_THREADS, (size_t)(3 * L * sizeof(float)), st>>>(
        w.Gp, w.dp, w.xf, N, (int)L, (int)w.Lp, w.Rpad, w.S, grad);
    return cudaGetLastError();
}

// Host side: pre-pass (digits + FP32 copy + transposed TF32 parts), the tensor-core sweep,
// the reduction, and the FP64 near-duplicate kernel. Requires L <= 320 and an sm_103 device.
inline int bt_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                     float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
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
    CUtensorMap mA, mB, mX;
    int rc;
    if ((rc = make_map(&mA, w.planes, false, w.Lp, 2 * w.Rpad, 128, err))) return rc;
    if ((rc = make_map(&mB, w.planes, false, w.Lp, 2 * w.Rpad, 64, err))) return rc;
    {
        // X^T parts: FP32 [2 Lp][Rpad]; boxes of 32 columns (128 bytes) x 64 atoms
        const cuuint64_t dims[2] = {(cuuint64_t)w.Rpad, (cuuint64_t)(2 * w.Lp)};
        const cuuint64_t strides[1] = {(cuuint64_t)(w.Rpad * 4)};
        const cuuint32_t box[2] = {32u, (cuuint32_t)BT_XCH};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, w.xT, dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            err = "cuTensorMapEncodeTiled (X^T) failed (" + std::to_string((int)r) + ")";
            return CLUSCO_ECUDA;
        }
    }
    const int64_t TA = w.Npad / TC_MA, TB = w.Npad / TC_MB;
    const int64_t JC = (TB + w.S - 1) / w.S;
    const int nkb = (int)(w.Lp / 64);
    const unsigned grid = (unsigned)(TA * w.S);
    e = cudaFuncSetAttribute(bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BT_SMEM);
    if (e == cudaSuccess) {
        prof_mark(PROF_ADJOINT, st);
        bwd_tc_kernel<<<grid, BT_THREADS, BT_SMEM, st>>>(mA, mB, mX, w.scales, w.G32, N, (int)L, (int)w.Lp, nkb,
                                                         w.Rpad, TB, w.S, JC, crmsd, grad_out, eps, w.Gp, w.dp,
                                                         w.nd_list, w.nd_count, w.nd_cap);
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
        err = std::string("tensor-core backward: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

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

// The adjoint: tensor-core recompute and contraction when the device and L allow it,
// else the CUDA-core path.
inline int backward_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                           float *grad, float eps, int form, void *ws, cudaStream_t st, std::string &err)
{
    if (L <= BT_MAXLP && tc_supported(CLUSCO_FORM_BF16_EXACT2, L) == CLUSCO_OK)
        return bt_launch(coords, N, L, grad_out, crmsd, grad, eps, ws, st, err);
    return backward_simt_launch(coords, N, L, grad_out, crmsd, grad, eps, form, ws, st, err);
}

}  // namespace clusco

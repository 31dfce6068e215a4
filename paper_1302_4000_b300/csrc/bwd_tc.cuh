// bwd_tc.cuh -- adjoint of the all-pairs matrix on the tensor cores (tcgen05).
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// One CTA (8 warps) owns one A tile I (40 models = 128 rows of the operand planes) and a
// contiguous range of B tiles J over the full square (every b != a in both orders, so the
// CTA owns its rows and needs no atomics). Tensor memory (512 columns) holds
//   cols [0, 192)        the tile covariance in three exact digit classes (hh, hl + lh, ll);
//   cols [192, 192 + Lp) the CTA's sum P.X over its column range (128 rows x Lp atoms,
//                        FP32), accumulated over the whole sweep.
// For every J:
//   1. GEMM1: the exact-digit covariance of the 40 x 20 tile (TMA -> 2-stage ring ->
//      tcgen05.mma kind::f16, as in the forward kernel, with hl and lh summed in one class:
//      |hl + lh| <= 2^15 per atom keeps the sum exact for L <= 512);
//   2. the warps read TMEM, assemble each 3x3 block (rows cyclic, as in the forward), take
//      Sigma from the FP32 fast path and the rotation from Horn's quaternion form, undo the
//      cyclic row order, and write w~ R as two TF32 parts (hi = rna(P), lo = rna(P - hi))
//      into a shared 128 x 64 operand in the 128-byte-swizzled K-major layout; pairs below
//      the near-duplicate threshold are queued for the FP64 direct kernel instead;
//   3. GEMM2: sum += P . X_J on tcgen05 kind::tf32 in three passes (hi.hi + hi.lo + lo.hi,
//      about 2^-21 relative per product), with X_J^T (atoms x 64) streamed by TMA from the
//      transposed hi / lo FP32 planes into the freed ring, in two atom chunks when Lp > 160.
// Rotations live only in shared memory. At the end the CTA reads the sum out of TMEM into
// its partial-gradient slice (negated); bwd_reduce_kernel adds the partials of the S column
// ranges, the diagonal term and the centring projection. Requires Lp = ceil(L/64)*64 <= 320.
#pragma once
#include "backward.cuh"
#include "pairs_tc.cuh"
#include "rotation.cuh"

namespace clusco {

constexpr int BT_THREADS = 256;
constexpr int BT_MAXLP = 320;
constexpr uint32_t BT_TMEM_COLS = 512;
constexpr uint32_t BT_D2 = 192;                            // first TMEM column of the P.X sum
constexpr size_t BT_RING = TC_STAGES * STAGE_BYTES_BF16;   // 96 KB; reused for X_J^T chunks
constexpr size_t BT_A2 = 2 * 128 * 64 * 4;                 // hi, lo: 64 KB
constexpr size_t BT_SMEM = 1024 + BT_RING + BT_A2;
static_assert(4 * 160 * 128 <= BT_RING, "an X^T chunk of 160 atoms fits the ring");

// Atoms per GEMM2 chunk: Lp itself up to 160, else Lp/2 (96, 128 or 160).
__host__ __device__ __forceinline__ int bt_chunk(int Lp) { return Lp <= 160 ? Lp : Lp / 2; }

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
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t done_bar;  // GEMM1 of the current J has landed in TMEM
    __shared__ __align__(8) uint64_t xt_bar;    // an X^T chunk has landed in the ring
    __shared__ __align__(8) uint64_t g2_bar;    // the GEMM2 MMAs of a chunk have finished
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float sB_scale[TC_MB * 3];
    __shared__ float sB_G32[TC_MB];
    __shared__ float dsum[TC_MA];

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase0 = smem_u32(smem);
    uint8_t *A2 = smem + BT_RING;  // [hi 32 KB][lo 32 KB]
    const uint32_t a2base = smem_u32(A2);
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
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        mbar_init(&xt_bar, 1);
        mbar_init(&g2_bar, 1);
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

    const int sp = warp & 3, g = warp >> 2;
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
    const int chunk = bt_chunk(Lp);
    const int nchunk = Lp / chunk;

    int64_t kbt = 0;        // GEMM1 K blocks issued so far (ring phase)
    uint32_t xt_count = 0;  // X^T chunks loaded so far (xt_bar and g2_bar phase)
    bool alive = true;
    for (int64_t J = J0; J < J1; ++J) {
        const int64_t jt = J - J0;
        const int64_t b_base = J * TC_MB;
        if (tid < TC_MB * 3) sB_scale[tid] = scales[(b_base + tid / 3) * 3 + tid % 3];
        if (tid < TC_MB) sB_G32[tid] = G32[b_base + tid];
        // ---- 1. GEMM1: tile covariance in three exact classes ----
        if (warp == 0 && lane == 0) {
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
            constexpr uint32_t id64 = make_idesc(128, 64, 1);
            for (int kb = 0; kb < nkb; ++kb) {
                const int64_t q = kbt + kb;
                const int s = (int)(q % TC_STAGES);
                const int64_t use = q / TC_STAGES;
                if (!mbar_wait(&full_bar[s], (uint32_t)(use & 1)) || *(volatile int *)&abort_flag) {
                    atomicExch(&abort_flag, 1);
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
        // The ring is free (GEMM1 has consumed it): start the first X^T chunk now, so that it
        // lands while the rotations are computed.
        auto load_chunk = [&](int ch) {
            const uint32_t blk = (uint32_t)chunk * 128u;
            mbar_arrive_expect_tx(&xt_bar, 4u * blk);
#pragma unroll
            for (int sp2 = 0; sp2 < 2; ++sp2)
#pragma unroll
                for (int kb2 = 0; kb2 < 2; ++kb2)
                    tma_load_2d(smem + (2 * sp2 + kb2) * blk, &mapX, &xt_bar, (int)(64 * J + 32 * kb2),
                                (int)(sp2 * Lp + ch * chunk));
        };
        if (warp == 0 && lane == 0) load_chunk(0);
        // ---- 2. rotations: w~ R of every pair into the TF32 hi / lo operand ----
        {
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
                const int bq = 3 * r + alpha;
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
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            const uint32_t off = a2_offset(32 * sp + 3 * mloc + i, 32 * g + 3 * bq + be);
                            const float v = P[3 * i + be];
                            const float vh = tf32_rna(v);
                            *reinterpret_cast<float *>(A2 + off) = vh;
                            *reinterpret_cast<float *>(A2 + 32768 + off) = tf32_rna(v - vh);
                        }
                }
            }
        }
        fence_proxy_async();  // the generic-proxy stores to A2 must be visible to tcgen05.mma
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- 3. GEMM2: sum += P . X_J in three TF32 passes, atom chunks ----
        if (warp == 0 && lane == 0) {
            const uint32_t id = make_idesc(128, chunk, 2);
            const uint32_t blk = (uint32_t)chunk * 128u;
            for (int ch = 0; ch < nchunk; ++ch) {
                if (ch > 0) load_chunk(ch);
                if (!mbar_wait(&xt_bar, xt_count & 1)) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + BT_D2 + (uint32_t)(ch * chunk);
#pragma unroll
                for (int kb2 = 0; kb2 < 2; ++kb2)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ahi = desc_sw128(a2base + kb2 * 16384 + 32 * k);
                        const uint64_t alo = desc_sw128(a2base + 32768 + kb2 * 16384 + 32 * k);
                        const uint64_t bhi = desc_sw128(sbase0 + kb2 * blk + 32 * k);
                        const uint64_t blo = desc_sw128(sbase0 + (2 + kb2) * blk + 32 * k);
                        // each chunk's first MMA of the sweep starts its columns from zero
                        mma_tf32(d, ahi, bhi, id, (jt == 0 && kb2 == 0 && k == 0) ? 0u : 1u);
                        mma_tf32(d, ahi, blo, id, 1u);
                        mma_tf32(d, alo, bhi, id, 1u);
                    }
                mma_commit(&g2_bar);
                // the ring is reused by the next chunk or the next J's GEMM1: wait for these MMAs
                const bool ok = mbar_wait(&g2_bar, xt_count & 1);
                ++xt_count;
                if (!ok) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*(volatile int *)&abort_flag) {
            alive = false;
            break;
        }
    }
    float *gp = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
    if (alive) {
        // ---- read the sum out of TMEM: warp (sp, g) takes lanes 32 sp.., half of the atoms ----
        const int half = Lp / 2;
        float *row = gp + (32 * sp + lane) * (int64_t)Lp;
        for (int c0 = g * half; c0 < (g + 1) * half; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * sp) << 16) + BT_D2 + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) row[c0 + j] = -v[j];
        }
        if (tid < TC_MA) dp[sidx * Npad + a_base + tid] = dsum[tid];
    } else {
        if (warp == 0 && lane == 0) {
            // drain (bounded) the loads this CTA issued before giving up
            for (int64_t q = (kbt > TC_STAGES ? kbt - TC_STAGES : 0); q < kbt; ++q)
                mbar_wait(&full_bar[q % TC_STAGES], (uint32_t)((q / TC_STAGES) & 1));
            mbar_wait(&xt_bar, xt_count & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BT_TMEM_COLS);
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
        // X^T parts: FP32 [2 Lp][Rpad]; boxes of 32 columns (128 bytes) x one atom chunk
        const cuuint64_t dims[2] = {(cuuint64_t)w.Rpad, (cuuint64_t)(2 * w.Lp)};
        const cuuint64_t strides[1] = {(cuuint64_t)(w.Rpad * 4)};
        const cuuint32_t box[2] = {32u, (cuuint32_t)bt_chunk((int)w.Lp)};
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
        bwd_tc_kernel<<<grid, BT_THREADS, BT_SMEM, st>>>(mA, mB, mX, w.scales, w.G32, N, (int)L, (int)w.Lp, nkb,
                                                         w.Rpad, TB, w.S, JC, crmsd, grad_out, eps, w.Gp, w.dp,
                                                         w.nd_list, w.nd_count, w.nd_cap);
        e = cudaGetLastError();
    }
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

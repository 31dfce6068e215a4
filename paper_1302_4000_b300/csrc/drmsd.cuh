// drmsd.cuh -- all-versus-all dRMSD (ClusCo, section "Algorithms", eq. 5): the RMS difference
// of two models' intra-model distance matrices over the K = L (L - 1) / 2 atom pairs i < j.
//
// Expanded, sum_k (d_a,k - d_b,k)^2 = |d_a|^2 + |d_b|^2 - 2 d_a . d_b: the Gram matrix of the
// N distance vectors over K, a dense contraction for the tensor cores, but one that cancels
// catastrophically for close models (|d|^2 / K, the mean squared distance, is thousands of
// A^2 against a dRMSD^2 of 1e-2 A^2 or less). The exact-digit form removes the cancellation:
// every distance is rounded to 16-bit fixed point with ONE scale q and ONE offset c0 for the
// whole ensemble, d ~ c0 + q n with |n| <= 32639, so that the differences of the rounded
// distances are q (n_a,k - n_b,k) exactly and only the integers n enter the contraction:
// n = 256 h + l with digits |h| <= 127, |l| <= 128 (exact in BF16), four digit-product
// classes hh, hl, lh, ll accumulated by tcgen05 in FP32. A class sum is exact while it has at
// most 1024 terms (1024 x 128^2 = 2^24), so the accumulator is drained every 1024 terms of K
// into an int64 sum per pair while the MMAs of the next 1024 terms run in the other half of
// tensor memory. Then D = sum_k (n_a,k - n_b,k)^2 = S_a + S_b - 2 G_ab exactly in int64 and
// dRMSD = q sqrt(2 D / (L (L - 1))). The one error is the rounding of the distances, at most
// q / 2 each, which moves dRMSD by at most q (the RMS norm's triangle inequality).
//
// Kernels: drmsd_range_kernel (largest distance of every model, hence q and c0),
// drmsd_quant_kernel (distances again, rounded, as two BF16 digit planes; or FP32 distances
// for the plain form), grouped_tiles_kernel (grouped tile order), drmsd_tc_kernel (the
// persistent tcgen05 contraction with the int64 drains and the eq. 5 epilogue) and
// drmsd_simt_kernel (the plain FP32 form: the squared differences summed directly on CUDA
// cores, compensated across K slabs).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "common.cuh"
#include "pairs_tc.cuh"
#include "prof.cuh"
#include "ptx.cuh"

namespace clusco {

constexpr int DR_MA = 128;            // A models per tile (TMEM lanes)
constexpr int DR_MB = 64;             // B models per tile ([B_h; B_l] = 128 MMA columns)
constexpr int DR_CHUNK_KB = 16;       // K blocks of 64 per exact FP32 chunk: 1024 terms
constexpr int DR_STAGES = 4;          // TMA ring depth (48 KB per stage)
constexpr int DR_EWARPS = 16;        // epilogue warps: 4 per TMEM lane quadrant, 16 B models each
constexpr int DR_THREADS = 64 + 32 * DR_EWARPS;  // warp 0 TMA, warp 1 MMA, warps 2-17 epilogue
constexpr int DR_GROUP = 8;           // tile rows per group of the schedule
constexpr int DR_NMAX = 32639;        // |n| <= 127 * 256 + 127
constexpr int DR_MAX_L = 4096;        // coordinates staged in shared memory (64 KB as float4)
constexpr size_t DR_SMEM = 1024 + (size_t)DR_STAGES * STAGE_BYTES_BF16;
static_assert(DR_SMEM <= 227 * 1024, "shared memory per CTA");

// ---- distance index: k = i (2L - i - 1) / 2 + (j - i - 1) for i < j ---------------------
__host__ __device__ __forceinline__ int64_t dr_row_start(int i, int L) { return (int64_t)i * (2 * L - i - 1) / 2; }

// Stage model a's coordinates in shared memory as float4 (x, y, z, 0), one 16-byte load per
// atom in the distance loops; true if all are finite (block-uniform).
__device__ __forceinline__ bool dr_stage(const float *__restrict__ coords, int64_t a, int L, float4 *xs)
{
    const float *x = coords + a * (int64_t)L * 3;
    bool ok = true;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const float4 v = make_float4(__ldg(x + 3 * t), __ldg(x + 3 * t + 1), __ldg(x + 3 * t + 2), 0.f);
        xs[t] = v;
        ok = ok && isfinite(v.x) && isfinite(v.y) && isfinite(v.z);
    }
    return __syncthreads_and(ok) != 0;
}

// Distances are enumerated by groups of DR_ROWS = 4 consecutive rows: warp w of a block takes
// the groups g = w, w + 8, ... and its lanes the columns j = 4 g + 1 + lane, + 32, ...; each
// staged atom j serves the group's four rows (one shared-memory load per four distances), the
// four squared distances take two passes of the packed FP32x2 pipe, stores are coalesced along
// each row, and no index is decoded. These kernels are issue-bound, hence the packing.
constexpr int DR_PRE_THREADS = 256;
constexpr int DR_ROWS = 4;

// The atoms of a row group by axis and row pair: x[p] = (x of row i0 + 2p, x of row i0 + 2p + 1).
// Rows past L - 2 repeat atom L - 1 (their distances are never stored).
struct DrRows {
    float2 x[2], y[2], z[2];
};

__device__ __forceinline__ DrRows dr_rows(const float4 *xs, int i0, int L)
{
    DrRows R;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float4 a = xs[min(i0 + 2 * p, L - 1)], b = xs[min(i0 + 2 * p + 1, L - 1)];
        R.x[p] = make_float2(a.x, b.x);
        R.y[p] = make_float2(a.y, b.y);
        R.z[p] = make_float2(a.z, b.z);
    }
    return R;
}

// d2[r] = squared distance of atom j to row atom i0 + r in FP32, rounded as
// fma(dx, dx, fma(dy, dy, dz * dz)) with each difference row - j rounded once (the contact test
// of the contact map overlap depends on this exact expression).
__device__ __forceinline__ void dr_dist2x4(const DrRows &R, const float4 &pj, float (&d2)[4])
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 xj = make_float2(pj.x, pj.x), yj = make_float2(pj.y, pj.y), zj = make_float2(pj.z, pj.z);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float2 dx = __ffma2_rn(xj, m1, R.x[p]), dy = __ffma2_rn(yj, m1, R.y[p]), dz = __ffma2_rn(zj, m1, R.z[p]);
        float2 q = __fmul2_rn(dz, dz);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dx, dx, q);
        d2[2 * p] = q.x;
        d2[2 * p + 1] = q.y;
    }
}

// One block per model: the largest intra-model distance (the square root of the largest squared
// distance, which is the largest rounded distance because sqrtf is monotone), folded into the
// ensemble's maximum (as the bits of a non-negative float, whose unsigned order is the numeric
// order), and the model's finiteness. Models with a non-finite coordinate take no part in the scale.
__global__ void __launch_bounds__(DR_PRE_THREADS) drmsd_range_kernel(const float *__restrict__ coords, int L,
                                                                     unsigned *__restrict__ dmax_bits,
                                                                     int *__restrict__ fin)
{
    extern __shared__ float4 xs[];
    __shared__ float red[DR_PRE_THREADS / 32];
    const int64_t a = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = DR_PRE_THREADS / 32;
    if (!dr_stage(coords, a, L, xs)) {
        if (threadIdx.x == 0) {
            fin[a] = 0;
            set_status(CLUSCO_ST_NONFINITE);
        }
        return;
    }
    // every d2 below is the squared distance of some atom pair of the model (or 0), so none
    // needs the masks that keep the quantiser to pairs i < j
    float m2 = 0.f;
    for (int i0 = DR_ROWS * warp; i0 < L - 1; i0 += DR_ROWS * NW) {
        const DrRows R = dr_rows(xs, i0, L);
        for (int j = i0 + 1 + lane; j < L; j += 32) {
            float d2[4];
            dr_dist2x4(R, xs[j], d2);
            m2 = fmaxf(m2, fmaxf(fmaxf(d2[0], d2[1]), fmaxf(d2[2], d2[3])));
        }
    }
    m2 = warp_max_f(m2);
    if (lane == 0) red[warp] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t = fmaxf(t, red[w]);
        atomicMax(dmax_bits, __float_as_uint(sqrtf(t)));
        fin[a] = 1;
    }
}

// The ensemble's rounding: d ~ c0 + q n, n in [-DR_NMAX, DR_NMAX] over [0, dmax].
struct DrScale {
    float q, c0, iq;
};
__device__ __forceinline__ DrScale dr_scale(unsigned dmax_bits)
{
    const float dmax = __uint_as_float(dmax_bits);
    DrScale s;
    const bool pos = dmax > 0.f && isfinite(dmax);
    s.q = pos ? dmax / (2.f * DR_NMAX) : 1.f;
    s.iq = pos ? (2.f * DR_NMAX) / dmax : 1.f;
    s.c0 = pos ? 0.5f * dmax : 0.f;
    return s;
}


// One block per padded model row. EXACT: digit planes (bf16, row a of the h plane and row
// Npad + a of the l plane, Kp wide, zero past K and for padding / non-finite models) and
// S[a] = sum n^2 (-1 marks a non-finite model). Plain form: FP32 distances [Npad][Kp]
// (NaN for a non-finite model, zero past K).
template <bool EXACT>
__global__ void __launch_bounds__(DR_PRE_THREADS) drmsd_quant_kernel(const float *__restrict__ coords, int64_t N,
                                                                     int L, int64_t Kp, int64_t Npad,
                                                                     const unsigned *__restrict__ dmax_bits,
                                                                     const int *__restrict__ fin,
                                                                     void *__restrict__ out, long long *__restrict__ S)
{
    extern __shared__ float4 xs[];
    constexpr int NW = DR_PRE_THREADS / 32;
    __shared__ long long red[NW];
    const int64_t a = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t K = (int64_t)L * (L - 1) / 2;
    const bool live = a < N && fin[a];
    __nv_bfloat16 *hrow = nullptr, *lrow = nullptr;
    float *frow = nullptr;
    if (EXACT) {
        hrow = reinterpret_cast<__nv_bfloat16 *>(out) + a * Kp;
        lrow = reinterpret_cast<__nv_bfloat16 *>(out) + (Npad + a) * Kp;
    } else {
        frow = reinterpret_cast<float *>(out) + a * Kp;
    }
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    if (!live) {
        const float fill = (a < N) ? __int_as_float(0x7fc00000) : 0.f;  // NaN rows for non-finite models
        for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) {
            if (EXACT) {
                hrow[k] = zero;
                lrow[k] = zero;
            } else {
                frow[k] = fill;
            }
        }
        if (EXACT && threadIdx.x == 0) S[a] = (a < N) ? -1 : 0;
        return;
    }
    dr_stage(coords, a, L, xs);
    const DrScale sc = dr_scale(EXACT ? *dmax_bits : 0u);
    long long s = 0;
    const float ofs = -sc.c0 * sc.iq;
    const float2 M2 = make_float2(12582912.f, 12582912.f), nM2 = make_float2(-12582912.f, -12582912.f);
    const float2 iq2 = make_float2(sc.iq, sc.iq), ofs2 = make_float2(ofs, ofs);
    const float2 r256 = make_float2(1.f / 256.f, 1.f / 256.f), m256 = make_float2(-256.f, -256.f);
    for (int i0 = DR_ROWS * warp; i0 < L - 1; i0 += DR_ROWS * NW) {
        const DrRows R = dr_rows(xs, i0, L);
        int64_t base[DR_ROWS];  // k = base + j in row i0 + r
#pragma unroll
        for (int r = 0; r < DR_ROWS; ++r) base[r] = dr_row_start(i0 + r, L) - (i0 + r) - 1;
        for (int j = i0 + 1 + lane; j < L; j += 32) {
            float d2[4];
            dr_dist2x4(R, xs[j], d2);
            if (EXACT) {
                // Conversions and the special-function unit run at a quarter of the FP32 rate, so
                // this path takes one sqrt.approx per distance (within 2 ulp; the rounding below
                // absorbs it) and does every rounding with the 1.5 * 2^23 shift on the FP32x2 pipe:
                // n = rint(clamp((d - c0) / q)), h = rint(n / 256) (|h| <= 127), l = n - 256 h
                // (|l| <= 128); h and l are small integers, so their BF16 encodings are the upper
                // halves of their FP32 encodings
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    float da, db;
                    asm("sqrt.approx.f32 %0, %1;" : "=f"(da) : "f"(d2[2 * p]));
                    asm("sqrt.approx.f32 %0, %1;" : "=f"(db) : "f"(d2[2 * p + 1]));
                    float2 x = __ffma2_rn(make_float2(da, db), iq2, ofs2);
                    x.x = fminf(fmaxf(x.x, -(float)DR_NMAX), (float)DR_NMAX);
                    x.y = fminf(fmaxf(x.y, -(float)DR_NMAX), (float)DR_NMAX);
                    const float2 t = __fadd2_rn(x, M2);
                    const float2 v = __fadd2_rn(t, nM2);
                    const float2 h = __fadd2_rn(__ffma2_rn(v, r256, M2), nM2);
                    const float2 l = __ffma2_rn(h, m256, v);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int r = 2 * p + u;
                        if (j <= i0 + r) continue;
                        const float hu = u ? h.y : h.x, lu = u ? l.y : l.x, tu = u ? t.y : t.x;
                        reinterpret_cast<unsigned short *>(hrow)[base[r] + j] = (unsigned short)(__float_as_uint(hu) >> 16);
                        reinterpret_cast<unsigned short *>(lrow)[base[r] + j] = (unsigned short)(__float_as_uint(lu) >> 16);
                        const int n = __float_as_int(tu) - 0x4B400000;
                        s += (long long)(n * n);  // n^2 <= 32639^2 < 2^31
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < DR_ROWS; ++r)
                    if (j > i0 + r) frow[base[r] + j] = sqrtf(d2[r]);
            }
        }
    }
    for (int64_t k = K + threadIdx.x; k < Kp; k += blockDim.x) {
        if (EXACT) {
            hrow[k] = zero;
            lrow[k] = zero;
        } else {
            frow[k] = 0.f;
        }
    }
    if (EXACT) {
        s = warp_sum_ll(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < NW; ++w) t += red[w];
            S[a] = t;
        }
    }
}

// Tile order of the persistent tensor-core kernels: tiles (I, J) of MA x MB models with pairs
// a < b, i.e. J >= jmin(I) = I MA / MB (MA and MB powers of two), in groups of `group` tile
// rows; within a group J ascending, then I. The grid's concurrent tiles then share a few A
// row panels and a few B panels, which stay in L2 while the CTAs stream K.
constexpr int TILE_ORDER_THREADS = 256;

__global__ void __launch_bounds__(TILE_ORDER_THREADS) grouped_tiles_kernel(int64_t TA, int64_t TB, int MA, int MB,
                                                                        int group, int2 *__restrict__ tiles)
{
    // one block per group, its threads over the columns J (a block-wide exclusive scan of the
    // columns' tile counts gives each column's first slot); jmin(I) = I MA / MB with MA / MB or
    // MB / MA a power of two (shifts, no 64-bit division)
    __shared__ int64_t s_off[TILE_ORDER_THREADS];
    __shared__ int64_t s_base;
    const int up = MA >= MB ? __ffs(MA / MB) - 1 : 0, dn = MB > MA ? __ffs(MB / MA) - 1 : 0;
    auto jmin = [&](int64_t I) { return (I << up) >> dn; };
    const int64_t I0 = (int64_t)blockIdx.x * group, I1 = min(TA, I0 + group);
    if (I0 >= TA) return;
    if (threadIdx.x == 0) {
        int64_t t0 = 0;  // tiles of the earlier groups
        for (int64_t I = 0; I < I0; ++I) t0 += TB - jmin(I);
        s_base = t0;
    }
    const int64_t J0 = jmin(I0);
    for (int64_t Jc = J0; Jc < TB; Jc += TILE_ORDER_THREADS) {
        const int64_t J = Jc + threadIdx.x;
        int64_t cnt = 0;
        if (J < TB)
            for (int64_t I = I0; I < I1 && jmin(I) <= J; ++I) ++cnt;
        s_off[threadIdx.x] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t run = s_base;
            for (int k = 0; k < TILE_ORDER_THREADS; ++k) {
                const int64_t v = s_off[k];
                s_off[k] = run;
                run += v;
            }
            s_base = run;
        }
        __syncthreads();
        if (J < TB) {
            int64_t t = s_off[threadIdx.x];
            for (int64_t I = I0; I < I1 && jmin(I) <= J; ++I) tiles[t++] = make_int2((int)I, (int)J);
        }
        __syncthreads();
    }
}

__host__ __device__ __forceinline__ int64_t dr_ntiles(int64_t TA, int64_t TB) { return TA * TB - TA * (TA - 1); }

__global__ void __launch_bounds__(DR_THREADS, 1)
    drmsd_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const int2 *__restrict__ tiles, int64_t ntiles, int64_t N, int L, int nkb, int64_t Npad,
                    const long long *__restrict__ S, const unsigned *__restrict__ dmax_bits, float *__restrict__ out)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[DR_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[DR_STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];   // a chunk's classes are in the buffer
    __shared__ __align__(8) uint64_t tempty_bar[2];  // the epilogue has read the buffer (one arrival per warp)
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase0 = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (nkb + DR_CHUNK_KB - 1) / DR_CHUNK_KB;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < DR_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], DR_EWARPS);
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
            for (int64_t t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x) {
                const int2 tj = tiles[t];
                for (int kb = 0; kb < nkb; ++kb, ++q) {
                    const int s = (int)(q % DR_STAGES);
                    const int64_t use = q / DR_STAGES;
                    if (q >= DR_STAGES && !mbar_wait_sleep(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                    uint8_t *st = smem + s * STAGE_BYTES_BF16;
                    mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES_BF16);
                    const int x = kb * 64;
                    tma_load_2d(st, &mapA, &full_bar[s], x, DR_MA * tj.x);
                    tma_load_2d(st + 16384, &mapA, &full_bar[s], x, (int)(Npad + DR_MA * tj.x));
                    tma_load_2d(st + 32768, &mapB, &full_bar[s], x, DR_MB * tj.y);
                    tma_load_2d(st + 40960, &mapB, &full_bar[s], x, (int)(Npad + DR_MB * tj.y));
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ================= MMA issuer: one TMEM buffer per 1024-term chunk =================
        if (lane == 0) {
            int64_t q = 0, c = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort_v; t += gridDim.x) {
                for (int ch = 0; ch < nch && ok; ++ch, ++c) {
                    const int buf = (int)(c & 1);
                    if (c >= 2 && !mbar_wait_sleep(&tempty_bar[buf], (uint32_t)(((c >> 1) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int kb1 = min(nkb, (ch + 1) * DR_CHUNK_KB);
                    for (int kb = ch * DR_CHUNK_KB; kb < kb1; ++kb, ++q) {
                        const int s = (int)(q % DR_STAGES);
                        if (!mbar_wait_sleep(&full_bar[s], (uint32_t)((q / DR_STAGES) & 1))) {
                            ok = false;
                            atomicExch(&abort_flag, 1);  // before the commit below wakes the epilogue
                            break;
                        }
                        tc_fence_after();
                        tc_issue_kblock<TC_EXACT2>(tmem + 256u * buf, sbase0 + s * STAGE_BYTES_BF16,
                                                   kb - ch * DR_CHUNK_KB);
                        mma_commit(&empty_bar[s]);
                    }
                    mma_commit(&tfull_bar[buf]);
                }
            }
            if (!ok) atomicExch(&abort_flag, 1);
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0)) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else {
        // ================= epilogue warps 2-17 =================
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (A models) and B models 16 g .. 16 g + 15
        const int sp = warp & 3, g = (warp - 2) >> 2;
        const DrScale sc = dr_scale(*dmax_bits);
        const float norm = 2.f / ((float)L * (float)(L - 1));
        int64_t c = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int2 tj = tiles[t];
            long long acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
            bool stop = false;
            for (int ch = 0; ch < nch; ++ch, ++c) {
                const int buf = (int)(c & 1);
                const bool okw = mbar_wait_sleep(&tfull_bar[buf], (uint32_t)((c >> 1) & 1));
                if (__any_sync(0xffffffffu, !okw || *abort_v)) {
                    atomicExch(&abort_flag, 1);
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t trow = tmem + 256u * buf + ((uint32_t)(32 * sp) << 16) + (uint32_t)(16 * g);
                // one class at a time (32 columns); each is an exact integer below 2^24 in magnitude:
                // G += 65536 hh + 256 (hl + lh) + ll
#pragma unroll
                for (int cls = 0; cls < 4; ++cls) {
                    uint32_t v[16];
                    tmem_ld16_issue(trow + 64 * cls, v);
                    tmem_wait_ld();
                    tmem_pin16(v);
                    const int sh = cls == 0 ? 16 : (cls == 3 ? 0 : 8);
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty_bar[buf]);
            }
            if (stop) break;
            // eq. 5 on the exact integer sums
            const int64_t a = (int64_t)DR_MA * tj.x + 32 * sp + lane;
            const int64_t b0 = (int64_t)DR_MB * tj.y + 16 * g;
            const long long Sb_l = (lane < 16 && b0 + lane < N) ? __ldg(S + b0 + lane) : 0;
            const long long Sa = (a < N) ? __ldg(S + a) : 0;
            const int64_t rowbase = a * N - a * (a + 1) / 2 - a - 1;  // condensed index - b
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const long long Sb = __shfl_sync(0xffffffffu, Sb_l, j);
                const int64_t b = b0 + j;
                if (a < b && b < N) {
                    float v;
                    if (Sa < 0 || Sb < 0) {
                        v = __int_as_float(0x7fc00000);
                    } else {
                        const long long D = Sa + Sb - 2 * acc[j];
                        v = sc.q * sqrtf((float)D * norm);
                    }
                    out[rowbase + b] = v;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (lane == 0 && *abort_v) {
            // a stopped CTA: the copies of the last armed stages may still be in flight (the MMA
            // issuer stopped waiting for them); they land before the CTA leaves (bounded waits)
            for (int64_t r = (q > DR_STAGES ? q - DR_STAGES : 0); r < q; ++r)
                mbar_wait(&full_bar[r % DR_STAGES], (uint32_t)((r / DR_STAGES) & 1));
        }
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
}

// Plain FP32 form: per 64 x 64 tile of model pairs, the squared differences of the FP32
// distances summed directly (no expansion, so no cancellation) on CUDA cores; each thread
// owns 4 x 4 pairs, 32-term partial sums per K slab are added with Kahan compensation.
constexpr int DRS_TILE = 64, DRS_KC = 32;

__global__ void __launch_bounds__(256) drmsd_simt_kernel(const float *__restrict__ Dk, int64_t N, int64_t Kp, int L,
                                                         int64_t T, float *__restrict__ out)
{
    __shared__ __align__(16) float As[DRS_KC][DRS_TILE];
    __shared__ __align__(16) float Bs[DRS_KC][DRS_TILE];
    int64_t I, J;
    tri_decode(blockIdx.x, T, &I, &J);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t a0 = I * DRS_TILE, b0 = J * DRS_TILE;
    float s[4][4], cmp[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) s[u][v] = cmp[u][v] = 0.f;
    for (int64_t k0 = 0; k0 < Kp; k0 += DRS_KC) {
        __syncthreads();
        for (int v = threadIdx.x; v < 2 * DRS_TILE * (DRS_KC / 4); v += 256) {
            const int which = v / (DRS_TILE * (DRS_KC / 4));
            const int r = v % (DRS_TILE * (DRS_KC / 4));
            const int m = r / (DRS_KC / 4), kq = r % (DRS_KC / 4);
            const float4 x = __ldg(reinterpret_cast<const float4 *>(Dk + ((which ? b0 : a0) + m) * Kp + k0) + kq);
            float(*dst)[DRS_TILE] = which ? Bs : As;
            dst[4 * kq + 0][m] = x.x;
            dst[4 * kq + 1][m] = x.y;
            dst[4 * kq + 2][m] = x.z;
            dst[4 * kq + 3][m] = x.w;
        }
        __syncthreads();
        float p[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) p[u][v] = 0.f;
#pragma unroll 8
        for (int kk = 0; kk < DRS_KC; ++kk) {
            const float4 av = *reinterpret_cast<const float4 *>(&As[kk][4 * ty]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tx]);
            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float d = ar[u] - br[v];
                    p[u][v] = fmaf(d, d, p[u][v]);
                }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float y = p[u][v] - cmp[u][v];
                const float t = s[u][v] + y;
                cmp[u][v] = (t - s[u][v]) - y;
                s[u][v] = t;
            }
    }
    const float norm = 2.f / ((float)L * (float)(L - 1));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t a = a0 + 4 * ty + u;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t b = b0 + 4 * tx + v;
            if (a < b && b < N) out[condensed_idx(a, b, N)] = sqrtf(s[u][v] * norm);
        }
    }
}

// ---- host side ----------------------------------------------------------

struct DrWs {
    void *planes = nullptr;  // EXACT: bf16 [2 Npad][Kp]; plain: FP32 [Npad][Kp]
    long long *S = nullptr;
    int *fin = nullptr;
    unsigned *dmax = nullptr;
    int2 *tiles = nullptr;
    int64_t Kp = 0, Npad = 0, ntiles = 0;
    size_t bytes = 0;
};

inline int drmsd_launch(const float *coords, int64_t N, int64_t L, float *out, bool exact, const DrWs &w,
                        cudaStream_t st, std::string &err)
{
    cudaError_t e = cudaSuccess;
    const size_t xsm = (size_t)L * sizeof(float4);
    if (xsm > 40 * 1024) {  // the static shared arrays count against the default 48 KB too
        e = cudaFuncSetAttribute(drmsd_range_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(drmsd_quant_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(drmsd_quant_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
        if (e != cudaSuccess) {
            err = std::string("dRMSD pre-pass shared memory: ") + cudaGetErrorString(e);
            return CLUSCO_ECUDA;
        }
    }
    e = cudaMemsetAsync(w.dmax, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        drmsd_range_kernel<<<(unsigned)N, DR_PRE_THREADS, xsm, st>>>(coords, (int)L, w.dmax, w.fin);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (exact)
            drmsd_quant_kernel<true><<<(unsigned)w.Npad, DR_PRE_THREADS, xsm, st>>>(coords, N, (int)L, w.Kp, w.Npad, w.dmax, w.fin,
                                                                        w.planes, w.S);
        else
            drmsd_quant_kernel<false><<<(unsigned)w.Npad, DR_PRE_THREADS, xsm, st>>>(coords, N, (int)L, w.Kp, w.Npad, w.dmax,
                                                                         w.fin, w.planes, w.S);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("dRMSD pre-pass: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    if (!exact) {
        const int64_t T = w.Npad / DRS_TILE;
        drmsd_simt_kernel<<<(unsigned)tri_tiles(T), 256, 0, st>>>(reinterpret_cast<const float *>(w.planes), N, w.Kp,
                                                                  (int)L, T, out);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            err = std::string("drmsd_simt_kernel: ") + cudaGetErrorString(e);
            return CLUSCO_ECUDA;
        }
        return CLUSCO_OK;
    }
    CUtensorMap mA, mB;
    int rc;
    if ((rc = make_map(&mA, w.planes, false, w.Kp, 2 * w.Npad, DR_MA, err))) return rc;
    if ((rc = make_map(&mB, w.planes, false, w.Kp, 2 * w.Npad, DR_MB, err))) return rc;
    const int64_t TA = w.Npad / DR_MA, TB = w.Npad / DR_MB;
    grouped_tiles_kernel<<<(unsigned)((TA + DR_GROUP - 1) / DR_GROUP), TILE_ORDER_THREADS, 0, st>>>(TA, TB, DR_MA, DR_MB,
                                                                                      DR_GROUP, w.tiles);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(drmsd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)DR_SMEM);
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned grid = (unsigned)std::min<int64_t>(w.ntiles, sms > 0 ? sms : 148);
        prof_mark(PROF_DRMSD, st);
        drmsd_tc_kernel<<<grid, DR_THREADS, DR_SMEM, st>>>(mA, mB, w.tiles, w.ntiles, N, (int)L, (int)(w.Kp / 64),
                                                           w.Npad, w.S, w.dmax, out);
        e = cudaGetLastError();
        prof_mark(PROF_DRMSD, st);
    }
    if (e != cudaSuccess) {
        err = std::string("drmsd_tc_kernel: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

}  // namespace clusco

// cmo.cuh -- all-versus-all contact map overlap (ClusCo, section "Algorithms", eq. 6 and eq. 7):
// contact maps C_ij = [ |x_i - x_j| < cutoff ] over the K = L (L - 1) / 2 atom pairs i < j, and
// S(A, B) = 100 * 2 n(A and B) / (n(A) + n(B)).
//
// n(A and B) = sum_k C_A,k C_B,k is the Gram matrix of the 0/1 maps: a dense contraction over K
// whose every partial sum is an integer below 2^24 (K < 2^24 for L <= 4096), so FP32
// accumulation is exact. The tensor-core form stores the maps as E4M3 bytes (1.0 = 0x38, 0 = 0)
// and contracts them with tcgen05 kind::f8f6f4 (twice the BF16 rate), 128 A models x 256 B
// models per tile, one accumulator per tile double-buffered in tensor memory: the counts, and
// hence the scores, are exact. The plain form packs the maps to bits and counts with AND and
// population count on CUDA cores.
//
// Kernels: cmo_map_kernel (the maps and n(A)), cmo_tc_kernel (persistent tcgen05 contraction
// with the eq. 7 epilogue), cmo_pack_kernel + cmo_popc_kernel (the plain form).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "common.cuh"
#include "drmsd.cuh"
#include "pairs_tc.cuh"
#include "prof.cuh"
#include "ptx.cuh"

namespace clusco {

constexpr int CM_MA = 128;                                 // A models per tile (TMEM lanes)
constexpr int CM_MB = 256;                                 // B models per tile (MMA N)
constexpr int CM_KB = 128;                                 // K elements (bytes) per stage row
constexpr int CM_STAGES = 4;
constexpr uint32_t CM_STAGE_BYTES = (CM_MA + CM_MB) * CM_KB;  // 48 KB
constexpr int CM_EWARPS = 16;                              // 4 per TMEM lane quadrant, 64 B models each
constexpr int CM_THREADS = 64 + 32 * CM_EWARPS;
constexpr int CM_GROUP = 8;
constexpr size_t CM_SMEM = 1024 + (size_t)CM_STAGES * CM_STAGE_BYTES;
constexpr unsigned char CM_ONE = 0x38;  // 1.0 in E4M3
static_assert(CM_SMEM <= 227 * 1024, "shared memory per CTA");

// One block per padded model row: the contact map as E4M3 bytes [Npad][Kp] (zero past K and for
// padding or non-finite models) and cnt[a] = n(A) (-1 marks a non-finite model). The contact test
// is d^2 < cutoff^2 in FP32 with d^2 = fma(dx, dx, fma(dy, dy, dz dz)).
__global__ void __launch_bounds__(DR_PRE_THREADS) cmo_map_kernel(const float *__restrict__ coords, int64_t N, int L,
                                                                 int64_t Kp, float cut2, uint8_t *__restrict__ map,
                                                                 int *__restrict__ cnt)
{
    extern __shared__ float4 xs[];
    constexpr int NW = DR_PRE_THREADS / 32;
    __shared__ int red[NW];
    const int64_t a = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t K = (int64_t)L * (L - 1) / 2;
    uint8_t *row = map + a * Kp;
    const bool live = a < N && dr_stage(coords, a, L, xs);
    if (!live) {
        for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) row[k] = 0;
        if (threadIdx.x == 0) {
            cnt[a] = (a < N) ? -1 : 0;
            if (a < N) set_status(CLUSCO_ST_NONFINITE);
        }
        return;
    }
    // scalar FP32 here: with one compare and one byte store per distance the packed pipe's
    // operand moves cost more than they save (measured). Only the first 32 columns of a row
    // group hold pairs i >= j to skip; the loop over the rest has no masks (7 % faster).
    int c = 0;
    for (int i0 = DR_ROWS * warp; i0 < L - 1; i0 += DR_ROWS * NW) {
        float4 pr[DR_ROWS];
        int64_t base[DR_ROWS];  // k = base + j in row i0 + r
#pragma unroll
        for (int r = 0; r < DR_ROWS; ++r) {
            pr[r] = xs[min(i0 + r, L - 1)];
            base[r] = dr_row_start(i0 + r, L) - (i0 + r) - 1;
        }
        uint8_t *rp[DR_ROWS];
#pragma unroll
        for (int r = 0; r < DR_ROWS; ++r) rp[r] = row + base[r];
        {
            const int j = i0 + 1 + lane;
            if (j < L) {
                const float4 pj = xs[j];
#pragma unroll
                for (int r = 0; r < DR_ROWS; ++r) {
                    if (j <= i0 + r) continue;
                    const float dx = pr[r].x - pj.x, dy = pr[r].y - pj.y, dz = pr[r].z - pj.z;
                    const bool in = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < cut2;
                    rp[r][j] = in ? CM_ONE : (uint8_t)0;
                    c += in ? 1 : 0;
                }
            }
        }
        for (int j = i0 + 33 + lane; j < L; j += 32) {
            const float4 pj = xs[j];
#pragma unroll
            for (int r = 0; r < DR_ROWS; ++r) {
                const float dx = pr[r].x - pj.x, dy = pr[r].y - pj.y, dz = pr[r].z - pj.z;
                const bool in = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < cut2;
                rp[r][j] = in ? CM_ONE : (uint8_t)0;
                c += in ? 1 : 0;
            }
        }
    }
    for (int64_t k = K + threadIdx.x; k < Kp; k += blockDim.x) row[k] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < NW; ++w) t += red[w];
        cnt[a] = t;
    }
}

// eq. 7 from the exact counts (0 where neither model has a contact; NaN for a non-finite model)
__device__ __forceinline__ float cmo_score(float nab, int na, int nb)
{
    if (na < 0 || nb < 0) return __int_as_float(0x7fc00000);
    const int s = na + nb;
    return s > 0 ? 200.f * nab / (float)s : 0.f;
}

__global__ void __launch_bounds__(CM_THREADS, 1)
    cmo_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const int2 *__restrict__ tiles, int64_t ntiles, int64_t N, int nkb, const int *__restrict__ cnt,
                  float *__restrict__ out)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[CM_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[CM_STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];   // the buffer holds a finished tile
    __shared__ __align__(8) uint64_t tempty_bar[2];  // the epilogue has read the buffer (one arrival per warp)
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase0 = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < CM_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], CM_EWARPS);
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
                    const int s = (int)(q % CM_STAGES);
                    const int64_t use = q / CM_STAGES;
                    if (q >= CM_STAGES && !mbar_wait_sleep(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                    uint8_t *st = smem + s * CM_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full_bar[s], CM_STAGE_BYTES);
                    const int x = kb * CM_KB;
                    tma_load_2d(st, &mapA, &full_bar[s], x, CM_MA * tj.x);
                    tma_load_2d(st + CM_MA * CM_KB, &mapB, &full_bar[s], x, CM_MB * tj.y);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ================= MMA issuer: one TMEM buffer per tile =================
        if (lane == 0) {
            constexpr uint32_t idesc = make_idesc(CM_MA, CM_MB, 0);  // e4m3 x e4m3 -> FP32
            int64_t q = 0, k = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort_v; t += gridDim.x, ++k) {
                const int buf = (int)(k & 1);
                if (k >= 2 && !mbar_wait_sleep(&tempty_bar[buf], (uint32_t)(((k >> 1) - 1) & 1))) {
                    ok = false;
                    atomicExch(&abort_flag, 1);
                    break;
                }
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb, ++q) {
                    const int s = (int)(q % CM_STAGES);
                    if (!mbar_wait_sleep(&full_bar[s], (uint32_t)((q / CM_STAGES) & 1))) {
                        ok = false;
                        atomicExch(&abort_flag, 1);  // before the commit below wakes the epilogue
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = sbase0 + s * CM_STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < CM_KB / 32; ++kk)
                        mma_f8(tmem + 256u * buf, desc_sw128(sb + 32 * kk), desc_sw128(sb + CM_MA * CM_KB + 32 * kk),
                               idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&empty_bar[s]);
                }
                mma_commit(&tfull_bar[buf]);
            }
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0)) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else {
        // ================= epilogue warps 2-17 =================
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (A models) and B models 64 g .. 64 g + 63
        const int sp = warp & 3, g = (warp - 2) >> 2;
        int64_t k = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
            const int2 tj = tiles[t];
            const int64_t a = (int64_t)CM_MA * tj.x + 32 * sp + lane;
            const int64_t b0 = (int64_t)CM_MB * tj.y + 64 * g;
            const int na = (a < N) ? __ldg(cnt + a) : 0;
            const int nb_lo = (b0 + lane < N) ? __ldg(cnt + b0 + lane) : 0;
            const int nb_hi = (b0 + 32 + lane < N) ? __ldg(cnt + b0 + 32 + lane) : 0;
            const int64_t rowbase = a * N - a * (a + 1) / 2 - a - 1;  // condensed index - b
            const int buf = (int)(k & 1);
            const bool okw = mbar_wait_sleep(&tfull_bar[buf], (uint32_t)((k >> 1) & 1));
            if (__any_sync(0xffffffffu, !okw || *abort_v)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            tc_fence_after();
            const uint32_t trow = tmem + 256u * buf + ((uint32_t)(32 * sp) << 16) + (uint32_t)(64 * g);
            uint32_t v0[32], v1[32];
            tmem_ld32_issue(trow, v0);
            tmem_ld32_issue(trow + 32, v1);
            tmem_wait_ld();
            tmem_pin32(v0);
            tmem_pin32(v1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty_bar[buf]);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int nb = __shfl_sync(0xffffffffu, nb_lo, j);
                const int64_t b = b0 + j;
                if (a < b && b < N) out[rowbase + b] = cmo_score(__uint_as_float(v0[j]), na, nb);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int nb = __shfl_sync(0xffffffffu, nb_hi, j);
                const int64_t b = b0 + 32 + j;
                if (a < b && b < N) out[rowbase + b] = cmo_score(__uint_as_float(v1[j]), na, nb);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (lane == 0 && *abort_v) {
            // a stopped CTA: the copies of the last armed stages may still be in flight (the MMA
            // issuer stopped waiting for them); they land before the CTA leaves (bounded waits)
            for (int64_t r = (q > CM_STAGES ? q - CM_STAGES : 0); r < q; ++r)
                mbar_wait(&full_bar[r % CM_STAGES], (uint32_t)((r / CM_STAGES) & 1));
        }
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
}

// ---- plain form: bit-packed maps, AND + population count on CUDA cores ----
// One thread packs 32 map bytes (two 16-byte loads) into one 32-bit word, bit t = byte t.
__global__ void cmo_pack_kernel(const uint8_t *__restrict__ map, int64_t nwords, uint32_t *__restrict__ bits)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
        const uint4 lo = __ldg(reinterpret_cast<const uint4 *>(map) + 2 * w);
        const uint4 hi = __ldg(reinterpret_cast<const uint4 *>(map) + 2 * w + 1);
        const uint32_t u[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        uint32_t r = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int by = 0; by < 4; ++by) r |= (((u[q] >> (8 * by)) & 0xffu) ? 1u : 0u) << (4 * q + by);
        bits[w] = r;
    }
}

constexpr int CMS_TILE = 64, CMS_KC = 32;  // 64 x 64 pairs per block, 32 words per slab

__global__ void __launch_bounds__(256) cmo_popc_kernel(const uint32_t *__restrict__ bits, int64_t N, int64_t W,
                                                       int64_t T, const int *__restrict__ cnt, float *__restrict__ out)
{
    __shared__ __align__(16) uint32_t As[CMS_KC][CMS_TILE];
    __shared__ __align__(16) uint32_t Bs[CMS_KC][CMS_TILE];
    int64_t I, J;
    tri_decode(blockIdx.x, T, &I, &J);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t a0 = I * CMS_TILE, b0 = J * CMS_TILE;
    int acc[4][4] = {};
    for (int64_t k0 = 0; k0 < W; k0 += CMS_KC) {
        __syncthreads();
        for (int v = threadIdx.x; v < 2 * CMS_TILE * (CMS_KC / 4); v += 256) {
            const int which = v / (CMS_TILE * (CMS_KC / 4));
            const int r = v % (CMS_TILE * (CMS_KC / 4));
            const int m = r / (CMS_KC / 4), kq = r % (CMS_KC / 4);
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(bits + ((which ? b0 : a0) + m) * W + k0) + kq);
            uint32_t(*dst)[CMS_TILE] = which ? Bs : As;
            dst[4 * kq + 0][m] = x.x;
            dst[4 * kq + 1][m] = x.y;
            dst[4 * kq + 2][m] = x.z;
            dst[4 * kq + 3][m] = x.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < CMS_KC; ++kk) {
            const uint4 av = *reinterpret_cast<const uint4 *>(&As[kk][4 * ty]);
            const uint4 bv = *reinterpret_cast<const uint4 *>(&Bs[kk][4 * tx]);
            const uint32_t ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] += __popc(ar[u] & br[w]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t a = a0 + 4 * ty + u;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int64_t b = b0 + 4 * tx + w;
            if (a < b && b < N) out[condensed_idx(a, b, N)] = cmo_score((float)acc[u][w], cnt[a], cnt[b]);
        }
    }
}

// ---- host side ----------------------------------------------------------

struct CmWs {
    uint8_t *map = nullptr;    // [Npad][Kp] E4M3 bytes
    uint32_t *bits = nullptr;  // plain form: [Npad][Kp / 32]
    int *cnt = nullptr;
    int2 *tiles = nullptr;
    int64_t Kp = 0, Npad = 0, ntiles = 0;
    size_t bytes = 0;
};

__host__ __device__ __forceinline__ int64_t cm_ntiles(int64_t TA, int64_t TB)
{
    int64_t n = 0;
    for (int64_t I = 0; I < TA; ++I) n += TB - I * CM_MA / CM_MB;
    return n;
}

inline int make_map_u8(CUtensorMap *m, void *base, int64_t Kp, int64_t rows, uint32_t box_rows, std::string &err)
{
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp};
    const cuuint32_t box[2] = {(cuuint32_t)CM_KB, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled (contact maps) failed (" + std::to_string((int)r) + ")";
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

inline int cmo_launch(const float *coords, int64_t N, int64_t L, float cutoff, float *out, bool tc, const CmWs &w,
                      cudaStream_t st, std::string &err)
{
    cudaError_t e = cudaSuccess;
    const size_t xsm = (size_t)L * sizeof(float4);
    if (xsm > 40 * 1024) e = cudaFuncSetAttribute(cmo_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
    if (e == cudaSuccess) {
        cmo_map_kernel<<<(unsigned)w.Npad, DR_PRE_THREADS, xsm, st>>>(coords, N, (int)L, w.Kp, cutoff * cutoff, w.map,
                                                                      w.cnt);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        err = std::string("contact maps: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    if (!tc) {
        const int64_t W = w.Kp / 32, T = w.Npad / CMS_TILE;
        cmo_pack_kernel<<<1184, 256, 0, st>>>(w.map, w.Npad * W, w.bits);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            cmo_popc_kernel<<<(unsigned)tri_tiles(T), 256, 0, st>>>(w.bits, N, W, T, w.cnt, out);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            err = std::string("cmo_popc_kernel: ") + cudaGetErrorString(e);
            return CLUSCO_ECUDA;
        }
        return CLUSCO_OK;
    }
    CUtensorMap mA, mB;
    int rc;
    if ((rc = make_map_u8(&mA, w.map, w.Kp, w.Npad, CM_MA, err))) return rc;
    if ((rc = make_map_u8(&mB, w.map, w.Kp, w.Npad, CM_MB, err))) return rc;
    const int64_t TA = w.Npad / CM_MA, TB = w.Npad / CM_MB;
    grouped_tiles_kernel<<<(unsigned)((TA + CM_GROUP - 1) / CM_GROUP), TILE_ORDER_THREADS, 0, st>>>(TA, TB, CM_MA, CM_MB,
                                                                                      CM_GROUP, w.tiles);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cmo_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CM_SMEM);
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned grid = (unsigned)std::min<int64_t>(w.ntiles, sms > 0 ? sms : 148);
        prof_mark(PROF_CMO, st);
        cmo_tc_kernel<<<grid, CM_THREADS, CM_SMEM, st>>>(mA, mB, w.tiles, w.ntiles, N, (int)(w.Kp / CM_KB), w.cnt, out);
        e = cudaGetLastError();
        prof_mark(PROF_CMO, st);
    }
    if (e != cudaSuccess) {
        err = std::string("cmo_tc_kernel: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    return CLUSCO_OK;
}

}  // namespace clusco

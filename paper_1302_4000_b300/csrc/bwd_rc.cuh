// bwd_rc.cuh -- adjoint of the all-pairs matrix on the tensor cores, every pair's rotation
// recomputed from the coordinates (nothing stored by the forward), L <= 1024 atoms.
//
// g_a = (sum_b w~_ab) a - sum_b (w~_ab R_ab) b,  w~ = w / (L max(c, eps))   (see backward.cuh)
//
// Work is split by A tile I (40 models = 128 operand rows), by a contiguous range of B tiles J
// over the full square (every b != a in both orders, so the owner of a row never needs another
// CTA's contributions), and by atom chunk: the sum P.X of a 128-row tile over L atoms is
// 128 x L FP32, more than tensor memory holds beside the covariance once L > 384, so each CTA
// accumulates the atoms of its own chunk (up to three 128-atom blocks; C chunks cover Lp).
// The C chunk CTAs of one (I, J range) form a thread-block cluster and share the per-pair work:
// CTA r of the cluster recomputes the covariance and the rotations of the tiles j = r, r + C, ..
// of the range, and every CTA copies the other tiles' rotation operands out of their owners'
// shared memory (distributed shared memory), so each covariance and each rotation is computed
// once per ordered pair, however many chunks L needs.
//
// Per CTA (608 threads; tensor memory: columns [0, 128) the covariance, [128, 128 + 128 q) the
// CTA's q atom blocks of the transposed sum):
//   warp 0 (TMA): for owned tiles the covariance operands (64-atom K blocks of X_I and X_J as
//     FP16 hi / lo parts, 2-stage ring, 128-byte swizzle);
//   warp 1 (MMA): GEMM1 of an owned tile: H = X_I X_J^T in three FP16 passes (hi.hi into
//     columns 0..63, hi.lo + lo.hi into 64..127 of one 128-column accumulator: A_hi against
//     the stacked [X_J,hi; X_J,lo] is one N = 128 MMA, A_lo against X_J,hi one N = 64 MMA);
//   warp 19 (TMA): the transposed parts X_J^T of the CTA's atom blocks (128 atoms x the tile's
//     64 rows), hi and lo halves in a 4-stage ring of half blocks, up to three ahead;
//   warp 18 (MMA): GEMM2 of every tile: sum^T += X_J^T P^T per atom block (M = 128 atoms,
//     N = 128 rows of the A tile, K = the tile's 64 rows, three FP16 passes: the hi half against
//     P_hi and P_lo, then the lo half against P_hi);
//   warps 2-17 (epilogue; four per TMEM lane quadrant, each the quadrant's 10 A models against 5
//     of the tile's 20 B models, two pairs per lane on the paired FP32 instructions): for owned
//     tiles, read the covariance out of tensor memory (then hand it back to GEMM1), assemble each
//     pair's 3 x 3 block (rows cyclic, as in the forward),
//     take Sigma (one Newton step from the forward's cRMSD) and the rotation R = dSigma/dM as the
//     top eigenvector of Horn's key matrix (Jacobi sweeps only at a numerically double root),
//     scale by w~, move the rows to the lanes that
//     own them with shuffles, and store the 128 x 64 operand P = w~ R as FP16 hi / lo parts
//     (K-major, 128-byte swizzle) into one of two slots, and send it to the other CTAs of the
//     cluster (one bulk copy into each peer's slot, shared memory to shared memory); the other
//     tiles' operands arrive the same way without any work of this CTA's threads. Pairs below
//     the near-duplicate threshold go to the FP64 direct kernel.
// Synchronisation between the CTAs of a cluster, per slot s (tile j uses slot j mod 2):
//   pfull[s] (local, 16 arrivals): this CTA has written its own tile's operand;
//   prx[s]   (1 arrival by the owner, plus the copy's bytes): a peer's operand has landed;
//   pfree[s][k mod 2] (C arrivals, a multicast tcgen05.commit from every CTA's MMA thread): every
//            CTA has finished GEMM2 of the slot's k-th tile (tile 2 k + s), so that the owner of
//            tile j + 2 may rewrite the slot and copy into every peer's. A parity wait is exact
//            only while the barrier is at most one phase away from the awaited one. With one
//            barrier per slot, the owner of tile j (which knows only that tiles up to j - C - 2
//            are done, from its wait before its previous tile j - C) could see tile j - 4's phase
//            still open for C = 3 and pass at once. With the slot's tiles split over two
//            barriers, the waited barrier's previous tile is j - 6, done for C <= 4, and its
//            next tile j + 2 cannot finish before tile j is written.
// Every wait is bounded. The CTAs of a cluster meet at cluster barriers after initialisation
// and, twice, before exit: after every MMA (and so every multicast commit) has completed and
// every copy has been issued, then after each CTA has waited for any copy still landing in it
// (only a stopped sweep can have one), so that no copy outlives its source or destination.
#pragma once
#include <cuda_fp16.h>

#include <cstdlib>

#include "bwd_rot.cuh"

namespace clusco {

// warp 0 covariance TMA, warp 1 covariance MMA (GEMM1), warps 2-17 epilogue, warp 18 contraction
// MMA (GEMM2), warp 19 X^T TMA
constexpr int RC_THREADS = 640;
constexpr int RC_G2WARP = 18;
constexpr int RC_XWARP = 19;
constexpr int RC_EPI = 16;  // epilogue warps: 4 per TMEM lane quadrant, 5 B models of a tile each
constexpr int RC_STAGES = 2;                          // GEMM1 ring
constexpr uint32_t RC_STAGE = 2 * 16384 + 2 * 8192;   // A_hi, A_lo (128 rows), B_hi, B_lo (64 rows) x 64 FP16
constexpr uint32_t RC_P = 2 * 16384;                  // operand P: hi, lo parts of 128 rows x 64 FP16
constexpr int RC_XSTAGES = 4;                         // X_J^T ring of half blocks
constexpr uint32_t RC_XHALF = 16384;                  // X_J^T hi or lo part of 128 atoms x 64 FP16
constexpr int RC_BLK = 128;                           // atoms per accumulator block (GEMM2 M)
constexpr int RC_MAXQ = 3;                            // accumulator blocks per CTA
constexpr int RC_MAXLP = 1024;
constexpr uint32_t RC_G2COL = 128;                    // first TMEM column of the transposed sum
constexpr size_t RC_SMEM = 1024 + RC_STAGES * RC_STAGE + 2 * RC_P + RC_XSTAGES * RC_XHALF;
static_assert(RC_SMEM + 1024 <= 227 * 1024, "shared memory per CTA");
static_assert((RC_MAXLP / RC_BLK + RC_MAXQ - 1) / RC_MAXQ <= 4, "the operand slots' barriers assume clusters of <= 4");

struct RcWs {
    float *xf = nullptr;      // [Rpad][Lp] centred FP32 (zero for padding and non-finite models)
    __half *x16 = nullptr;    // [2][Rpad][Lp] FP16 hi / lo parts of xf 2^kx, atoms contiguous
    __half *xT = nullptr;     // [2][Lp][Rpad] the same parts transposed
    float *G32 = nullptr;     // [Npad] sum of squares of the centred coordinates
    float *Gp = nullptr;      // [Smax][Rpad][Lp] partial gradients (one slice per column range)
    float *dp = nullptr;      // [Smax C][Npad] partial row sums of w~
    long long *nd_list = nullptr;
    unsigned long long *nd_count = nullptr;
    unsigned *scl = nullptr;  // max |centred x|, max |w| (float bits)
    int64_t Lp = 0, Npad = 0, Rpad = 0, Smax = 1, C = 1, q = 1, nblk = 1, nd_cap = 0;
    size_t bytes = 0;
};

// Atom chunks: 128-atom blocks, at most RC_MAXQ per CTA, spread evenly over C CTAs.
inline void rc_chunks(int64_t Lp, int64_t &nblk, int64_t &C, int64_t &q)
{
    nblk = (Lp + RC_BLK - 1) / RC_BLK;
    C = (nblk + RC_MAXQ - 1) / RC_MAXQ;
    q = (nblk + C - 1) / C;
}

// Column ranges per A tile: about four waves of 148 SMs, and at most twice that plus two (the
// workspace's partial slices); the launch picks the count within that bound that fills whole waves
// of the clusters the device can hold at once (rc_pick_splits).
inline int64_t rc_splits(int64_t TA, int64_t TB, int64_t C)
{
    int64_t S = (4 * 148 + TA * C - 1) / (TA * C);
    if (S > TB) S = TB;
    return S < 1 ? 1 : S;
}

inline int64_t rc_max_splits(int64_t TA, int64_t TB, int64_t C)
{
    const int64_t S = 2 * rc_splits(TA, TB, C) + 2;
    return S > TB ? TB : S;
}

// The count of column ranges that minimises waves x tiles per range for `resident` work groups
// (clusters, or CTAs without clusters) at a time, each group taking one (A tile, range); a 1 %
// charge per range stands for the reduction of the partial slices.
inline int64_t rc_pick_splits(int64_t TA, int64_t TB, int64_t Smax, int64_t resident)
{
    if (resident < 1) resident = 1;
    int64_t best = 1;
    double best_cost = 1e300;
    for (int64_t S = 1; S <= Smax; ++S) {
        const double waves = (double)((TA * S + resident - 1) / resident);
        const double cost = waves * (double)((TB + S - 1) / S) * (1.0 + 0.01 * (double)S);
        if (cost < best_cost) {
            best_cost = cost;
            best = S;
        }
    }
    return best;
}

inline RcWs carve_rc(void *base, int64_t N, int64_t L)
{
    RcWs w;
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
    rc_chunks(w.Lp, w.nblk, w.C, w.q);
    w.Smax = rc_max_splits(w.Npad / TC_MA, w.Npad / TC_MB, w.C);
    w.xf = (float *)take(sizeof(float) * w.Rpad * w.Lp);
    w.x16 = (__half *)take(sizeof(__half) * 2 * w.Rpad * w.Lp);
    w.xT = (__half *)take(sizeof(__half) * 2 * w.Lp * w.Rpad);
    w.G32 = (float *)take(sizeof(float) * w.Npad);
    w.Gp = (float *)take(sizeof(float) * w.Smax * w.Rpad * w.Lp);
    w.dp = (float *)take(sizeof(float) * w.Smax * w.C * w.Npad);
    const int64_t P = N * (N - 1) / 2;
    w.nd_cap = nd_cap_for(P);
    w.nd_list = (long long *)take(sizeof(long long) * 2 * w.nd_cap);
    w.nd_count = (unsigned long long *)take(sizeof(unsigned long long));
    w.scl = (unsigned *)take(2 * sizeof(unsigned));
    w.bytes = off;
    return w;
}

// Centred FP32 rows in the tensor-core row layout, the sum of squares G32 per model, and the
// largest |centred coordinate| over the finite models. A model with a non-finite coordinate
// gets zero rows and G32 = NaN: every pair it is in has a NaN cRMSD, which routes the pair to
// the FP64 direct kernel (which propagates the NaN into both gradients), and its zero rows
// keep the contraction of every other model finite. Grid: ceil(Npad/8) blocks of 256 threads.
__global__ void __launch_bounds__(256) rc_prepass_kernel(const float *__restrict__ coords, int64_t N, int L, int Lp,
                                                         int64_t Npad, float *__restrict__ xf,
                                                         float *__restrict__ G32, unsigned *__restrict__ xmax)
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
        if (lane == 0) G32[a] = 0.f;
        return;
    }
    const float *x = coords + a * (int64_t)L * 3;
    float mu[3];
    bool finite;
    model_centroid(x, L, lane, mu, &finite);
    if (!finite) {
        for (int ax = 0; ax < 3; ++ax) zero_row(r0 + ax);
        if (lane == 0) G32[a] = __int_as_float(0x7fc00000);
        return;
    }
    float m = 0.f, g = 0.f;
    for (int i = lane; i < Lp; i += 32)
        for (int ax = 0; ax < 3; ++ax) {
            const float v = (i < L) ? (x[3 * i + ax] - mu[ax]) : 0.f;
            xf[(r0 + ax) * Lp + i] = v;
            m = fmaxf(m, fabsf(v));
            g = fmaf(v, v, g);
        }
    m = warp_max_f(m);
    g = warp_sum_f(g);
    if (lane == 0) {
        G32[a] = g;
        if (m > 0.f) atomicMax(xmax, __float_as_uint(m));
    }
}

// FP16 parts (hi = rn(v), lo = rn(v - hi)) of v = xf 2^kx, both in the row layout (x16, the
// covariance operands) and transposed (xT, the contraction's X_J^T). 32 x 32 tiles through
// shared memory; grid (Rpad / 32, Lp / 32) blocks of 256 threads.
__global__ void __launch_bounds__(256) rc_split_kernel(const float *__restrict__ xf, int64_t Rpad, int Lp,
                                                       const unsigned *__restrict__ xmax, __half *__restrict__ x16,
                                                       __half *__restrict__ xT)
{
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const float sx = exp2i(fp16_scale_exp(__uint_as_float(*xmax)));
    for (int k = ty; k < 32; k += 8) {
        const float v = xf[(r0 + k) * Lp + i0 + tx] * sx;
        t[k][tx] = v;
        const __half hi = __float2half_rn(v);
        x16[(r0 + k) * Lp + i0 + tx] = hi;
        x16[(Rpad + r0 + k) * Lp + i0 + tx] = __float2half_rn(v - __half2float(hi));
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const float v = t[tx][k];
        const __half hi = __float2half_rn(v);
        xT[(int64_t)(i0 + k) * Rpad + r0 + tx] = hi;
        xT[((int64_t)Lp + i0 + k) * Rpad + r0 + tx] = __float2half_rn(v - __half2float(hi));
    }
}

// The pair's rotation from its normalised covariance m: Sigma_hat by one Newton step on m's
// quartic from s0 (the forward's cRMSD gives it: L c^2 = (G_A + G_B)(1 - Sigma_hat)), then the top
// eigenvector of Horn's key matrix at that Sigma_hat (the symmetric adjugate of K - Sigma_hat I,
// its column of largest diagonal entry, as a unit quaternion). The closed form dSigma/dM loses
// accuracy already where P'(Sigma) < 0.08 Sigma^3 (about 1 % of the pairs of a decoy ensemble,
// and every warp round that holds one would run the slow path); the adjugate holds down to
// P' ~ 1e-4 Sigma^3, below which no pair of these ensembles falls, and needs no orthogonality
// polish (a unit quaternion gives an orthogonal matrix to rounding). Below that the caller takes
// Jacobi sweeps (rotation_robust).
//
// Two pairs at once, one in each half of a float2, on the paired FP32 instructions (two IEEE
// operations per instruction): the same steps as rc_rotation, so that each lane carries two
// independent chains and half the instructions per pair. Selections, reciprocals and the
// validity tests stay per pair.
// Horn's adjugate column for one of the two pairs (h = 0: .x, 1: .y): the column of the
// largest diagonal entry, and whether that entry clears tol * lam^3.
__device__ __forceinline__ bool horn_pick(const float (&d)[10], float lam, float tol, float q[4])
{
    // d: d00 d01 d02 d03 d11 d12 d13 d22 d23 d33
    float best = fabsf(d[0]);
    q[0] = d[0], q[1] = d[1], q[2] = d[2], q[3] = d[3];
    if (fabsf(d[4]) > best) {
        best = fabsf(d[4]);
        q[0] = d[1], q[1] = d[4], q[2] = d[5], q[3] = d[6];
    }
    if (fabsf(d[7]) > best) {
        best = fabsf(d[7]);
        q[0] = d[2], q[1] = d[5], q[2] = d[7], q[3] = d[8];
    }
    if (fabsf(d[9]) > best) {
        best = fabsf(d[9]);
        q[0] = d[3], q[1] = d[6], q[2] = d[8], q[3] = d[9];
    }
    return best > tol * fabsf(lam) * lam * lam && isfinite(best);
}

__device__ __forceinline__ void rc_rotation2(const float2 m[9], float2 s0, float2 R[9], bool &okx, bool &oky)
{
    // minors3 and the invariants I1, det, I2
    float2 mn[9];
    mn[0] = dif2(m[3], m[7], m[4], m[6]);
    mn[1] = dif2(m[3], m[8], m[5], m[6]);
    mn[2] = dif2(m[4], m[8], m[5], m[7]);
    mn[3] = dif2(m[0], m[7], m[1], m[6]);
    mn[4] = dif2(m[0], m[8], m[2], m[6]);
    mn[5] = dif2(m[1], m[8], m[2], m[7]);
    mn[6] = dif2(m[0], m[4], m[1], m[3]);
    mn[7] = dif2(m[0], m[5], m[2], m[3]);
    mn[8] = dif2(m[1], m[5], m[2], m[4]);
    const float2 det = fma2(m[2], mn[0], sub2(mul2(m[0], mn[2]), mul2(m[1], mn[1])));
    float2 I2 = mul2(mn[0], mn[0]), I1 = mul2(m[0], m[0]);
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        I2 = fma2(mn[k], mn[k], I2);
        I1 = fma2(m[k], m[k], I1);
    }
    // one Newton step on x^4 - 2 I1 x^2 - 8 det x + (I1^2 - 4 I2), skipped near a double root
    const float2 c2 = mul2(bc2(-2.f), I1), c1 = mul2(bc2(-8.f), det);
    const float2 c0 = fma2(I1, I1, mul2(bc2(-4.f), I2));
    const float2 sq = mul2(s0, s0);
    const float2 P = fma2(add2(sq, c2), sq, fma2(c1, s0, c0));
    const float2 dP = fma2(fma2(bc2(4.f), sq, mul2(bc2(2.f), c2)), s0, c1);
    const float2 lim = mul2(bc2(8e-3f), mul2(sq, s0));
    float2 s = s0;
    if (dP.x > lim.x) s.x -= __fdividef(P.x, dP.x);
    if (dP.y > lim.y) s.y -= __fdividef(P.y, dP.y);
    // Horn's key matrix K(m) - s I and its symmetric adjugate
    const float2 tr = add2(add2(m[0], m[4]), m[8]);
    const float2 a00 = sub2(tr, s);
    const float2 a11 = sub2(sub2(mul2(bc2(2.f), m[0]), tr), s);
    const float2 a22 = sub2(sub2(mul2(bc2(2.f), m[4]), tr), s);
    const float2 a33 = sub2(sub2(mul2(bc2(2.f), m[8]), tr), s);
    const float2 a01 = sub2(m[7], m[5]), a02 = sub2(m[2], m[6]), a03 = sub2(m[3], m[1]);
    const float2 a12 = add2(m[1], m[3]), a13 = add2(m[2], m[6]), a23 = add2(m[5], m[7]);
    const float2 t0 = dif2(a00, a11, a01, a01), t1 = dif2(a00, a12, a01, a02), t2 = dif2(a00, a13, a01, a03);
    const float2 t3 = dif2(a01, a12, a11, a02), t4 = dif2(a01, a13, a11, a03), t5 = dif2(a02, a13, a12, a03);
    const float2 u1 = dif2(a02, a23, a03, a22), u2 = dif2(a02, a33, a03, a23), u3 = dif2(a12, a23, a13, a22);
    const float2 u4 = dif2(a12, a33, a13, a23), u5 = dif2(a22, a33, a23, a23);
    float2 dd[10];
    dd[0] = fma2(a13, u3, dif2(a11, u5, a12, u4));   // d00
    dd[1] = sub2(mul2(a02, u4), fma2(a01, u5, mul2(a03, u3)));  // d01
    dd[2] = fma2(a33, t3, dif2(a13, t5, a23, t4));   // d02
    dd[3] = sub2(mul2(a22, t4), fma2(a12, t5, mul2(a23, t3)));  // d03
    dd[4] = fma2(a03, u1, dif2(a00, u5, a02, u2));   // d11
    dd[5] = sub2(mul2(a23, t2), fma2(a03, t5, mul2(a33, t1)));  // d12
    dd[6] = fma2(a23, t1, dif2(a02, t5, a22, t2));   // d13
    dd[7] = fma2(a33, t0, dif2(a03, t4, a13, t2));   // d22
    dd[8] = sub2(mul2(a12, t2), fma2(a02, t4, mul2(a23, t0)));  // d23
    dd[9] = fma2(a22, t0, dif2(a02, t3, a12, t1));   // d33
    float dx[10], dy[10], qx[4], qy[4];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        dx[k] = dd[k].x;
        dy[k] = dd[k].y;
    }
    okx = horn_pick(dx, s.x, 1e-4f, qx);
    oky = horn_pick(dy, s.y, 1e-4f, qy);
    float2 q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = make_float2(qx[k], qy[k]);
    const float2 n2 = fma2(q[3], q[3], fma2(q[2], q[2], fma2(q[1], q[1], mul2(q[0], q[0]))));
    const float2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
    const float2 w = mul2(q[0], inv), x = mul2(q[1], inv), y = mul2(q[2], inv), z = mul2(q[3], inv);
    const float2 ww = mul2(w, w), xx = mul2(x, x), yy = mul2(y, y), zz = mul2(z, z);
    const float2 two = bc2(2.f);
    R[0] = sub2(add2(ww, xx), add2(yy, zz));
    R[1] = mul2(two, dif2(x, y, w, z));
    R[2] = mul2(two, fma2(x, z, mul2(w, y)));
    R[3] = mul2(two, fma2(x, y, mul2(w, z)));
    R[4] = sub2(add2(ww, yy), add2(xx, zz));
    R[5] = mul2(two, dif2(y, z, w, x));
    R[6] = mul2(two, dif2(x, z, w, y));
    R[7] = mul2(two, fma2(y, z, mul2(w, x)));
    R[8] = sub2(add2(ww, zz), add2(xx, yy));
}

// Cyclic assembly (see assemble_block) of round r's block on the window of one epilogue warp: the
// 15 covariance columns of 5 B models (rounds 0 and 1 hold B models t and 3 + t of the window; a
// lane whose model falls past the window gets a zero block and has no pair). The round is a
// compile-time constant so that every index into V is static.
template <int r>
__device__ __forceinline__ void rc_assemble5(const float (&V)[15], int alpha, int mloc, float blk[9])
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

// Round r's rotation rows to the lanes that own them, on a 5-model window. Lane (mloc, t) computed
// the pair of window model 3 r + t; its rotation rows arrive cyclically (row k of send is axis
// (t + k) mod 3 of the A model), already scaled. Lane (mloc, alpha) needs row alpha of the three
// pairs: from lane t it takes that lane's row (alpha - t) mod 3, so in shuffle k every lane sends
// row k and receives from lane (alpha - k) mod 3. The rows land in v at columns 3 (3 r + t) + beta.
template <int r>
__device__ __forceinline__ void rc_scatter5(const float (&send)[9], int alpha, int mloc, float (&v)[17])
{
    float rcv[3][3];
#pragma unroll
    for (int be = 0; be < 3; ++be) rcv[0][be] = send[be];
#pragma unroll
    for (int k = 1; k <= 2; ++k) {
        const int src = (3 * mloc + (alpha + 3 - k) % 3) & 31;
#pragma unroll
        for (int be = 0; be < 3; ++be) rcv[k][be] = __shfl_sync(0xffffffffu, send[3 * k + be], src);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        if (3 * r + t >= 5) continue;  // past the five B models of this window
        const int k = (alpha + 3 - t) % 3;
#pragma unroll
        for (int be = 0; be < 3; ++be) v[3 * (3 * r + t) + be] = sel3(k, rcv[0][be], rcv[1][be], rcv[2][be]);
    }
}

__device__ __forceinline__ void tmem_pin1(uint32_t &r) { asm volatile("" : "+r"(r)); }

// FP16 hi / lo parts of two floats, as the bits of two half2
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t &hb, uint32_t &lb)
{
    const __half2 hh = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    hb = *reinterpret_cast<const uint32_t *>(&hh);
    lb = *reinterpret_cast<const uint32_t *>(&ll);
}

__global__ void __launch_bounds__(RC_THREADS, 1)
    bwd_rc_kernel(const __grid_constant__ CUtensorMap mapXA, const __grid_constant__ CUtensorMap mapXB,
                  const __grid_constant__ CUtensorMap mapTh, const __grid_constant__ CUtensorMap mapTl,
                  const float *__restrict__ G32, int64_t N, int L, int Lp, int nkb, int64_t Rpad, int64_t TB,
                  int64_t S, int64_t JC, int C, int q, int nblk, int CS, const float *__restrict__ crmsd,
                  const float *__restrict__ wvec, float eps, const unsigned *__restrict__ scl,
                  float *__restrict__ Gp, float *__restrict__ dp, long long *__restrict__ nd_list,
                  unsigned long long *__restrict__ nd_count, int64_t nd_cap)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[RC_STAGES];    // GEMM1 ring: K block landed
    __shared__ __align__(8) uint64_t empty_bar[RC_STAGES];   // GEMM1 ring: K block consumed
    __shared__ __align__(8) uint64_t done1_bar;              // GEMM1 of an owned tile is in TMEM
    __shared__ __align__(8) uint64_t tfree_bar;              // the epilogue has read it (8 arrivals)
    __shared__ __align__(8) uint64_t pfull_bar[2];           // an owned tile's operand is written (8 arrivals)
    __shared__ __align__(8) uint64_t prx_bar[2];             // a peer's operand has landed (1 arrival + bytes)
    __shared__ __align__(8) uint64_t pfree_bar[2][2];        // every CTA finished GEMM2 of a tile (CS arrivals)
    __shared__ __align__(8) uint64_t xfull_bar[RC_XSTAGES];  // an X^T half block landed
    __shared__ __align__(8) uint64_t xempty_bar[RC_XSTAGES]; // GEMM2 has finished reading it
    __shared__ __align__(8) uint64_t d2_bar;                 // every GEMM2 MMA of this CTA has completed
    __shared__ __align__(8) uint64_t g1end_bar;              // every GEMM1 MMA of this CTA has completed
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int64_t g2_done, g2_seen;                     // GEMM2 tiles committed / operands waited for
    __shared__ float dpart[4][TC_MA];  // row sums of w~ per A model, one slot per column quarter

    // 1024-byte aligned in the shared window; indexing smem_raw keeps the pointer in the shared
    // address space
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *RING = smem;
    uint8_t *PS = smem + RC_STAGES * RC_STAGE;  // two operand slots of RC_P bytes
    uint8_t *XT = PS + 2 * RC_P;                // RC_XSTAGES X^T half blocks of RC_XHALF bytes
    const uint32_t ringbase = smem_u32(RING), pbase = smem_u32(PS), xtbase = smem_u32(XT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t cl = blockIdx.x / C;  // the cluster (CS = C) or the group of C chunk CTAs
    const int chunk = CS > 1 ? (int)cluster_ctarank() : (int)(blockIdx.x % C);
    const int64_t Npad = Rpad / 32 * 10;
    // slice-major: the clusters of a wave share one column range (its B and X^T panels stay in
    // L2 while they sweep it together) and differ in A tile (8,192 x 500: DRAM reads 2.01 -> 1.02
    // GB, 3.83 -> 3.71 ms per launch)
    const int64_t I = cl % (Npad / TC_MA), sidx = cl / (Npad / TC_MA);
    const int64_t J0 = sidx * JC, J1 = (J0 + JC < TB) ? J0 + JC : TB;
    const int64_t a_base = I * TC_MA;
    const int blk0 = chunk * q;
    const int nb = (nblk - blk0 < q) ? nblk - blk0 : q;  // this CTA's atom blocks (>= 1)
    // who does what: in a cluster (CS = C) CTA r owns the tiles j = r mod C and writes its own
    // row-sum slice; without one (CS = 1) every chunk CTA owns every tile, and chunk 0 alone
    // writes the row sums and queues the near-duplicate pairs
    const int crank = CS > 1 ? chunk : 0;
    const bool lead = CS > 1 || chunk == 0;
    const int64_t dslice = sidx * C + chunk;  // non-lead CTAs write zeros there

    if (J0 >= J1) {  // an empty column range still owns its (zero) partial slices
        float *gp = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
        for (int e = tid; e < 128 * nb * RC_BLK; e += RC_THREADS) {
            const int r = e / (nb * RC_BLK), at = blk0 * RC_BLK + e % (nb * RC_BLK);
            if (at < Lp) gp[(int64_t)r * Lp + at] = 0.f;
        }
        if (tid < TC_MA) dp[dslice * Npad + a_base + tid] = 0.f;
        return;  // every CTA of the cluster shares the range, so all of them return here
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < RC_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < RC_XSTAGES; ++s) {
            mbar_init(&xfull_bar[s], 1);
            mbar_init(&xempty_bar[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&pfull_bar[s], RC_EPI);
            mbar_init(&prx_bar[s], 1);
            mbar_init(&pfree_bar[s][0], (uint32_t)CS);
            mbar_init(&pfree_bar[s][1], (uint32_t)CS);
        }
        mbar_init(&done1_bar, 1);
        mbar_init(&tfree_bar, RC_EPI);
        mbar_init(&d2_bar, 1);
        mbar_init(&g1end_bar, 1);
        abort_flag = 0;
        g2_done = g2_seen = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    // the operand slots' pad rows (lanes 30, 31 of each quadrant) stay zero for the whole sweep
    for (int e = tid; e < (int)(2 * RC_P / 16); e += RC_THREADS)
        reinterpret_cast<float4 *>(PS)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (CS > 1) cluster_sync_all();  // every peer's barriers are initialised before any remote access
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int64_t nJ = J1 - J0;
    volatile int *abort_v = &abort_flag;
    auto owned = [&](int64_t j) { return CS == 1 || (int)(j % CS) == crank; };
    // stages armed by the covariance producer (warp 0, lane 0) and by the X^T producer (warp 19,
    // lane 0)
    int64_t q1 = 0, cx = 0;

    if (warp == 0) {
        // ================= TMA producer: covariance operands of the owned tiles =================
        if (lane == 0) {
            tma_prefetch_desc(&mapXA);
            tma_prefetch_desc(&mapXB);
            bool ok = true;
            auto g1_loads = [&](int64_t J) {
                for (int kb = 0; kb < nkb && ok; ++kb, ++q1) {
                    const int s = (int)(q1 % RC_STAGES);
                    const int64_t use = q1 / RC_STAGES;
                    if (q1 >= RC_STAGES && !mbar_wait_sleep(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = RING + s * RC_STAGE;
                    mbar_arrive_expect_tx(&full_bar[s], RC_STAGE);
                    const int x = kb * 64;
                    tma_load_2d(st, &mapXA, &full_bar[s], x, (int)(128 * I));
                    tma_load_2d(st + 16384, &mapXA, &full_bar[s], x, (int)(Rpad + 128 * I));
                    tma_load_2d(st + 32768, &mapXB, &full_bar[s], x, (int)(64 * J));
                    tma_load_2d(st + 40960, &mapXB, &full_bar[s], x, (int)(Rpad + 64 * J));
                }
            };
            // in the order of the GEMM1 thread's consumption
            for (int64_t j = crank; j < nJ && ok && !*abort_v; j += CS) g1_loads(J0 + j);
            if (!ok) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else if (warp == 1 || warp == RC_G2WARP) {
        // ================= MMA issuers: covariance GEMM1 (warp 1), contraction GEMM2 (warp 18) =================
        // Two threads, so that GEMM1 of the next owned tile goes out as soon as the epilogue has read
        // the current covariance, whatever operand GEMM2 is waiting for; each thread's commits track
        // its own MMAs, and they touch disjoint tensor memory and shared memory.
        if (lane == 0) {
            int64_t q1 = 0, xc = 0, ko = 0, gd = 0, seen = 0;
            int po0 = 0, po1 = 0;  // own operands written into slot 0 / 1
            int rx0 = 0, rx1 = 0;  // peer operands received into slot 0 / 1
            bool ok = true;
            constexpr uint32_t id128 = make_idesc(128, 128, 0);  // FP16 operands
            constexpr uint32_t id64 = make_idesc(128, 64, 0);
            const uint16_t mask = (uint16_t)((1u << CS) - 1u);
            auto g1 = [&]() {
                for (int kb = 0; kb < nkb && ok; ++kb, ++q1) {
                    const int s = (int)(q1 % RC_STAGES);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((q1 / RC_STAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = ringbase + s * RC_STAGE;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ah = desc_sw128(sb + 32 * k), al = desc_sw128(sb + 16384 + 32 * k);
                        const uint64_t bb = desc_sw128(sb + 32768 + 32 * k);  // [X_J,hi; X_J,lo], 128 rows
                        mma_f16(tmem + 0, ah, bb, id128, (kb > 0 || k > 0) ? 1u : 0u);  // hh | hl
                        mma_f16(tmem + 64, al, bb, id64, 1u);                          // + lh (X_J,hi rows)
                    }
                    mma_commit(&empty_bar[s]);
                }
                mma_commit(&done1_bar);
            };
            auto g2 = [&](int64_t jj) {
                const int s = (int)(jj & 1);
                bool got;
                if (owned(jj)) {
                    got = mbar_wait(&pfull_bar[s], (uint32_t)((s ? po1 : po0) & 1));
                    if (s)
                        ++po1;
                    else
                        ++po0;
                } else if (s) {
                    got = mbar_wait(&prx_bar[1], (uint32_t)(rx1 & 1));
                    ++rx1;
                } else {
                    got = mbar_wait(&prx_bar[0], (uint32_t)(rx0 & 1));
                    ++rx0;
                }
                seen = jj + 1;
                if (!got) {
                    ok = false;
                    return;
                }
                tc_fence_after();
                const uint32_t pb = pbase + s * RC_P;
                for (int bl = 0; bl < nb && ok; ++bl, ++xc) {
                    const uint32_t d = tmem + RC_G2COL + (uint32_t)(bl * 128);
                    // the block's hi half (X_J,hi against P_hi and P_lo), then its lo half (X_J,lo
                    // against P_hi), each from its own stage of the ring
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const int64_t hh = 2 * xc + part;
                        const int st = (int)(hh % RC_XSTAGES);
                        if (!mbar_wait(&xfull_bar[st], (uint32_t)((hh / RC_XSTAGES) & 1))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t xb = xtbase + st * RC_XHALF;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t xd = desc_sw128(xb + 32 * k);
                            const uint64_t phi = desc_sw128(pb + 32 * k), plo = desc_sw128(pb + RC_P / 2 + 32 * k);
                            if (part == 0) {
                                // each block's first MMA of the sweep starts its columns from zero
                                mma_f16(d, xd, phi, id128, (jj == 0 && k == 0) ? 0u : 1u);
                                mma_f16(d, xd, plo, id128, 1u);
                            } else {
                                mma_f16(d, xd, phi, id128, 1u);
                            }
                        }
                        mma_commit(&xempty_bar[st]);
                    }
                }
                if (!ok) return;
                uint64_t *pf = &pfree_bar[s][(jj >> 1) & 1];
                if (CS > 1)
                    mma_commit_multicast(pf, mask);
                else
                    mma_commit(pf);
                gd = jj + 1;
            };
            if (warp == 1) {
                // GEMM1 of the next owned tile as soon as the epilogue has read the current covariance,
                // so that it runs under the epilogue's rotations
                for (int64_t j = crank; j < nJ && ok && !*abort_v; j += CS) {
                    if (ko > 0 && !mbar_wait_sleep(&tfree_bar, (uint32_t)((ko - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    g1();
                    ++ko;
                }
            } else {
                for (int64_t j = 0; j < nJ && ok && !*abort_v; ++j) g2(j);
            }
            // also on abort: fires once everything this thread issued has completed
            uint64_t *endb = (warp == 1) ? &g1end_bar : &d2_bar;
            mma_commit(endb);
            if (!mbar_wait(endb, 0)) ok = false;
            if (!ok) atomicExch(&abort_flag, 1);
            if (warp == RC_G2WARP) {
                g2_done = gd;
                g2_seen = seen;
            }
        }
        __syncwarp();
    } else if (warp == RC_XWARP) {
        // ================= TMA producer: X^T half blocks of every tile =================
        // half block h: block h / 2 of the sweep (tile h / (2 nb), atom block of this CTA's chunk),
        // part h mod 2 (hi, lo), into stage h mod RC_XSTAGES once GEMM2 has finished reading the
        // stage's previous half block; so up to three half blocks load while GEMM2 reads the fourth
        if (lane == 0) {
            tma_prefetch_desc(&mapTh);
            tma_prefetch_desc(&mapTl);
            const int64_t nxh = 2 * nJ * nb;
            bool ok = true;
            for (int64_t h = 0; h < nxh && ok && !*abort_v; ++h) {
                const int st = (int)(h % RC_XSTAGES);
                if (h >= RC_XSTAGES && !mbar_wait_sleep(&xempty_bar[st], (uint32_t)(((h / RC_XSTAGES) - 1) & 1))) {
                    ok = false;
                    break;
                }
                // the tile's 64 operand rows x 128 atoms; atoms past Lp read as zeros
                const int64_t t = h >> 1;
                const int x = (int)(64 * (J0 + t / nb)), y = (blk0 + (int)(t % nb)) * RC_BLK;
                mbar_arrive_expect_tx(&xfull_bar[st], RC_XHALF);
                tma_load_2d(XT + st * RC_XHALF, (h & 1) ? &mapTl : &mapTh, &xfull_bar[st], x, y);
                cx = h + 1;
            }
            if (!ok) atomicExch(&abort_flag, 1);
        }
        __syncwarp();
    } else {
        // ================= epilogue warps 2..17 =================
        // Warp (sp, g, hw): TMEM lane quadrant sp (= warp mod 4, the quadrant its tcgen05.ld
        // reaches), i.e. the 10 A models of that quadrant, against the five B models
        // 10 g + 5 hw .. + 4 of every owned tile (covariance columns 32 g + 15 hw .. + 14).
        const int etid = tid - 64, ew = warp - 2;
        const int sp = warp & 3, g = (ew >> 2) & 1, hw = ew >> 3;
        const int mloc = lane / 3, alpha = lane - 3 * (lane / 3);
        const int la = 10 * sp + mloc;
        const int64_t a = a_base + la;
        const bool lane_ok = lane < 30 && a < N;
        const float fL = (float)L;
        const float Ga = lane_ok ? G32[a] : 0.f;
        const int kx = fp16_scale_exp(__uint_as_float(scl[0]));
        const int kp = fp16_scale_exp(__uint_as_float(scl[1]) / (fL * fmaxf(CLUSCO_NEARDUP, eps)));
        const float sP = exp2i(kp), ixs = exp2i(-kx);
        const uint32_t tcol = tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)(32 * g);
        float csum = 0.f;
        int64_t ko = 0;
        bool alive = true;
        // forward outputs, weights and sums of squares of this lane's two pairs of an owned tile
        // (B models alpha and 3 + alpha of the window)
        float cpre[2], wpre[2], gpre[2];
        bool val[2];
        // condensed index of (a, b): above the diagonal rowA + b, below it b (2N - b - 1) / 2 - b - 1 + a
        const int64_t rowA = a * (2 * N - a - 1) / 2 - a - 1;
        auto fetch = [&](int64_t jt) {
            const int64_t b0 = (J0 + jt) * TC_MB + 10 * g + 5 * hw;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int bq = 3 * r + alpha;
                const int64_t b = b0 + bq;
                val[r] = jt < nJ && lane_ok && bq < 5 && b < N && b != a;
                cpre[r] = 0.f;
                wpre[r] = 0.f;
                gpre[r] = 0.f;
                if (val[r]) {
                    const int64_t idx = a < b ? rowA + b : b * (2 * N - b - 1) / 2 - b - 1 + a;
                    cpre[r] = __ldg(crmsd + idx);
                    wpre[r] = __ldg(wvec + idx);
                    gpre[r] = __ldg(G32 + b);
                }
            }
        };
        const int64_t jstep = CS;  // owned tiles are crank, crank + CS, ...
        fetch(crank);
        for (int64_t j = crank; j < nJ; j += jstep) {
            const int s = (int)(j & 1);
            uint8_t *slot = PS + s * RC_P;
            const int64_t b0 = (J0 + j) * TC_MB + 10 * g + 5 * hw;
            const float cx = cpre[0], cy = cpre[1], wx = wpre[0], wy = wpre[1], gx = gpre[0], gy = gpre[1];
            const bool vx = val[0], vy = val[1];
            float V[15];
            // warp-uniform: tcgen05.ld below is a warp-wide instruction
            bool fail = __any_sync(0xffffffffu, !mbar_wait_sleep(&done1_bar, (uint32_t)(ko & 1)));
            ++ko;
            if (!fail) {
                tc_fence_after();
                // the window's 15 columns of hh | hl (columns 0..63) and of hl + lh (64..127); window 1
                // starts at column 15, so it takes one column and the 16 from column 16
                // one class at a time (16 registers in flight, not 32)
                uint32_t u[16];
                if (hw == 0) {
                    tmem_ld16_issue(tcol, u);
                    tmem_wait_ld();
                    tmem_pin16(u);
#pragma unroll
                    for (int jj = 0; jj < 15; ++jj) V[jj] = __uint_as_float(u[jj]);
                    tmem_ld16_issue(tcol + 64, u);
                    tmem_wait_ld();
                    tmem_pin16(u);
#pragma unroll
                    for (int jj = 0; jj < 15; ++jj) V[jj] += __uint_as_float(u[jj]);
                } else {
                    uint32_t e0 = tmem_ld1_issue(tcol + 15);
                    tmem_ld16_issue(tcol + 16, u);
                    tmem_wait_ld();
                    tmem_pin1(e0);
                    tmem_pin16(u);
                    V[0] = __uint_as_float(e0);
#pragma unroll
                    for (int jj = 0; jj < 14; ++jj) V[jj + 1] = __uint_as_float(u[jj]);
                    e0 = tmem_ld1_issue(tcol + 79);
                    tmem_ld16_issue(tcol + 80, u);
                    tmem_wait_ld();
                    tmem_pin1(e0);
                    tmem_pin16(u);
                    V[0] += __uint_as_float(e0);
#pragma unroll
                    for (int jj = 0; jj < 14; ++jj) V[jj + 1] += __uint_as_float(u[jj]);
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < 15; ++jj) V[jj] = 0.f;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tfree_bar);  // TMEM columns 0..127 may be overwritten now
            // the lane's two pairs (rounds 0 and 1 of the window) in the two halves of the paired
            // instructions
            float bx[9], by[9];
            rc_assemble5<0>(V, alpha, mloc, bx);
            rc_assemble5<1>(V, alpha, mloc, by);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float c = h ? cy : cx, w = h ? wy : wx;
                const bool vr = h ? vy : vx;
                const int64_t b = b0 + 3 * h + alpha;
                if (lead && vr && !(c >= CLUSCO_NEARDUP) && w != 0.f && a < b) {
                    const unsigned long long slot_nd = atomicAdd(nd_count, 1ull);
                    if ((int64_t)slot_nd < nd_cap) {
                        nd_list[2 * slot_nd] = a;
                        nd_list[2 * slot_nd + 1] = b;
                    }
                }
            }
            const float coefx = (vx && cx >= CLUSCO_NEARDUP && wx != 0.f) ? __fdividef(wx, fL * fmaxf(cx, eps)) : 0.f;
            const float coefy = (vy && cy >= CLUSCO_NEARDUP && wy != 0.f) ? __fdividef(wy, fL * fmaxf(cy, eps)) : 0.f;
            csum += coefx + coefy;
            float sx[9], sy[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) sx[e] = sy[e] = 0.f;
            if ((coefx != 0.f || coefy != 0.f) && !fail) {
                const float igx = __fdividef(1.f, Ga + gx), igy = __fdividef(1.f, Ga + gy);
                const float2 nrm = make_float2(2.f * igx * ixs * ixs, 2.f * igy * ixs * ixs);
                float2 m[9], R[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) m[e] = mul2(make_float2(bx[e], by[e]), nrm);
                // Sigma_hat from the forward's cRMSD: L c^2 = (G_A + G_B)(1 - Sigma_hat)
                const float2 s0 = make_float2(fmaf(-fL * cx * cx, igx, 1.f), fmaf(-fL * cy * cy, igy, 1.f));
                bool okx, oky;
                rc_rotation2(m, s0, R, okx, oky);
                const float csx = coefx * sP, csy = coefy * sP;
                // a pair without a coefficient (near-duplicate, padding) has no rotation: the half it
                // occupied may hold anything, so select, do not multiply by zero
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    sx[e] = coefx != 0.f ? csx * R[e].x : 0.f;
                    sy[e] = coefy != 0.f ? csy * R[e].y : 0.f;
                }
                if ((!okx && coefx != 0.f) || (!oky && coefy != 0.f)) {  // a numerically double root
                    float mh[9], Rh[9];
                    if (!okx && coefx != 0.f) {
#pragma unroll
                        for (int e = 0; e < 9; ++e) mh[e] = m[e].x;
                        rotation_robust(mh, Rh);
#pragma unroll
                        for (int e = 0; e < 9; ++e) sx[e] = csx * Rh[e];
                    }
                    if (!oky && coefy != 0.f) {
#pragma unroll
                        for (int e = 0; e < 9; ++e) mh[e] = m[e].y;
                        rotation_robust(mh, Rh);
#pragma unroll
                        for (int e = 0; e < 9; ++e) sy[e] = csy * Rh[e];
                    }
                }
            }
            float v[17];
            v[15] = v[16] = 0.f;  // window 1's columns 30, 31: the group's two zero rows
            rc_scatter5<0>(sx, alpha, mloc, v);
            rc_scatter5<1>(sy, alpha, mloc, v);
            // the next owned tile's forward outputs and weights: their latency hides behind this
            // tile's operand store and the wait for the next covariance
            fetch(j + jstep);
            // the slot's previous tile (j - 2) must be done in every CTA's GEMM2
            if (!fail && j >= 2) {
                const int64_t k = (j >> 1) - 1;  // tile j - 2 is the slot's k-th tile
                fail = !mbar_wait_sleep(&pfree_bar[s][k & 1], (uint32_t)((k >> 1) & 1));
            }
            if (!fail && lane < 30) {
                // row 32 sp + lane of the operand, columns 32 g + 15 hw .. of its 64: 16-byte chunks at
                // (chunk ^ (row mod 8)), FP16 hi / lo parts. Window 0 fills chunk 4 g and the first
                // seven columns of chunk 4 g + 1, window 1 that chunk's last column and chunks
                // 4 g + 2, 4 g + 3 (2-byte stores where the two windows share a word)
                const int row = 32 * sp + lane;
                uint8_t *hb = slot + row * 128, *lb = hb + RC_P / 2;
                auto choff = [&](int chunk) { return ((chunk ^ (row & 7)) & 7) << 4; };
                if (hw == 0) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split_h2(v[2 * e], v[2 * e + 1], h[e], l[e]);
                    *reinterpret_cast<uint4 *>(hb + choff(4 * g)) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(lb + choff(4 * g)) = make_uint4(l[0], l[1], l[2], l[3]);
                    const int o = choff(4 * g + 1);
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        split_h2(v[8 + 2 * e], v[9 + 2 * e], h[e], l[e]);
                        *reinterpret_cast<uint32_t *>(hb + o + 4 * e) = h[e];
                        *reinterpret_cast<uint32_t *>(lb + o + 4 * e) = l[e];
                    }
                    split_h2(v[14], 0.f, h[3], l[3]);
                    *reinterpret_cast<uint16_t *>(hb + o + 12) = (uint16_t)(h[3] & 0xffffu);
                    *reinterpret_cast<uint16_t *>(lb + o + 12) = (uint16_t)(l[3] & 0xffffu);
                } else {
                    uint32_t h[4], l[4];
                    const int o = choff(4 * g + 1);
                    split_h2(v[0], 0.f, h[0], l[0]);
                    *reinterpret_cast<uint16_t *>(hb + o + 14) = (uint16_t)(h[0] & 0xffffu);
                    *reinterpret_cast<uint16_t *>(lb + o + 14) = (uint16_t)(l[0] & 0xffffu);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) split_h2(v[1 + 8 * q + 2 * e], v[2 + 8 * q + 2 * e], h[e], l[e]);
                        *reinterpret_cast<uint4 *>(hb + choff(4 * g + 2 + q)) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4 *>(lb + choff(4 * g + 2 + q)) = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                }
            }
            // generic-proxy stores to the slot must be visible to tcgen05.mma and to the bulk copies
            fence_proxy_async();
            __syncwarp();
            if (lane == 0 && !fail) mbar_arrive(&pfull_bar[s]);
            if (named_bar_or(1, 32 * RC_EPI, fail || *abort_v)) {
                alive = false;
                break;
            }
            if (CS > 1 && ew == 0 && lane == 0) {
                // every warp has written its part: send the operand to the other CTAs of the cluster,
                // whose slot s is free (pfree above covers their GEMM2 of tile j - 2)
                const uint32_t sbar = smem_u32(&prx_bar[s]), sdst = pbase + s * RC_P;
                for (int rk = 0; rk < CS; ++rk) {
                    if (rk == crank) continue;
                    const uint32_t rbar = mapa_shared(sbar, (uint32_t)rk);
                    mbar_arrive_expect_tx_remote(rbar, RC_P);
                    bulk_copy_to_peer(mapa_shared(sdst, (uint32_t)rk), slot, RC_P, rbar);
                }
            }
        }
        // row sums of w~ per A model: the three lanes of a model, then one slot per column quarter
        // (ew / 4), added in a fixed order below, so that the sums do not depend on warp timing
        float cs3 = csum + __shfl_down_sync(0xffffffffu, csum, 1) + __shfl_down_sync(0xffffffffu, csum, 2);
        if (lane < 30 && alpha == 0) dpart[ew >> 2][la] = cs3;
        {  // every epilogue warp, stopped or not, meets the others here once
            const bool ok3 = alive && mbar_wait_sleep(&d2_bar, 0);
            alive = !named_bar_or(1, 32 * RC_EPI, !ok3 || *abort_v);
        }
        if (alive) {
            tc_fence_after();
            // read the transposed sum out of TMEM: warp (sp, q = ew / 4) takes TMEM lanes 32 sp..
            // (atoms) and the q-th quarter of each block's 128 columns (rows of the A tile); undo
            // both scales
            const float ix = exp2i(-kx), ip = exp2i(-kp);
            float *gbase = Gp + (sidx * Rpad + 128 * I) * (int64_t)Lp;
            const int r0 = 32 * (ew >> 2);
            // 16 columns at a time: a 32-column load here, with the sweep's state still live,
            // made the register allocator spill inside the tile loop
#pragma unroll 1
            for (int bl = 0; bl < nb; ++bl) {
                const int atom = (blk0 + bl) * RC_BLK + 32 * sp + lane;
                float *gcol = gbase + (int64_t)r0 * Lp + atom;
#pragma unroll 1
                for (int hc = 0; hc < 32; hc += 16) {
                    uint32_t vv[16];
                    tmem_ld16_issue(tmem + ((uint32_t)(32 * sp) << 16) + RC_G2COL + (uint32_t)(bl * 128 + r0 + hc), vv);
                    tmem_wait_ld();
                    tmem_pin16(vv);
                    if (atom < Lp) {
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            gcol[(int64_t)(hc + jj) * Lp] = -(__uint_as_float(vv[jj]) * ix) * ip;
                    }
                }
            }
            if (etid < TC_MA)
                dp[dslice * Npad + a_base + etid] =
                    lead ? ((dpart[0][etid] + dpart[1][etid]) + dpart[2][etid]) + dpart[3][etid] : 0.f;
        } else {
            atomicExch(&abort_flag, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (lane == 0 && *abort_v) {
        // a stopped CTA: the TMA copies of the last armed stages may still be in flight (the MMA
        // issuers stopped waiting for them); they land before the CTA leaves (bounded waits)
        if (warp == 0)
            for (int64_t r = (q1 > RC_STAGES ? q1 - RC_STAGES : 0); r < q1; ++r)
                mbar_wait(&full_bar[r % RC_STAGES], (uint32_t)((r / RC_STAGES) & 1));
        if (warp == RC_XWARP)
            for (int64_t r = (cx > RC_XSTAGES ? cx - RC_XSTAGES : 0); r < cx; ++r)
                mbar_wait(&xfull_bar[r % RC_XSTAGES], (uint32_t)((r / RC_XSTAGES) & 1));
    }
    if (CS > 1) {
        // every CTA has issued all its copies; on a stopped sweep, operands a peer may still be
        // copying into this CTA (at most the two tiles after the last one whose GEMM2 this CTA
        // committed) land before the cluster dissolves, so that no copy outlives its source or
        // destination (bounded waits; nothing is in flight on a completed sweep)
        cluster_sync_all();
        if (tid == 64 && *abort_v) {
            int64_t rx0 = 0, rx1 = 0;
            for (int64_t jj = 0; jj < g2_seen; ++jj)
                if (!owned(jj)) {
                    if (jj & 1)
                        ++rx1;
                    else
                        ++rx0;
                }
            for (int64_t jj = g2_seen; jj < g2_done + 2 && jj < nJ; ++jj) {
                if (owned(jj)) continue;
                if (jj & 1)
                    mbar_wait(&prx_bar[1], (uint32_t)(rx1++ & 1));
                else
                    mbar_wait(&prx_bar[0], (uint32_t)(rx0++ & 1));
            }
        }
        __syncthreads();
        cluster_sync_all();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
}

inline bool rc_supported(int64_t L) { return (L + 63) / 64 * 64 <= RC_MAXLP; }

// Host side, in two parts. rc_prepare: the pre-pass (centred rows, FP16 parts in both layouts,
// the two scales), which reads only the coordinates and the weights, so that it may run beside
// the forward. rc_sweep: the tensor-core sweep (clusters of C CTAs when the device can co-schedule
// them, else C independent CTAs that each recompute the rotations), the reduction of the partial
// slices, and the FP64 kernel of the near-duplicate pairs, after the forward and the pre-pass.
// Requires L <= 1024 and an sm_103 device.
inline int rc_prepare(const float *coords, int64_t N, int64_t L, const float *grad_out, void *ws, cudaStream_t st,
                      std::string &err)
{
    const RcWs w = carve_rc(ws, N, L);
    const int64_t P = N * (N - 1) / 2;
    cudaError_t e = cudaMemsetAsync(w.scl, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.nd_count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        rc_prepass_kernel<<<(unsigned)((w.Npad + 7) / 8), 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.xf,
                                                                        w.G32, w.scl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        rc_split_kernel<<<dim3((unsigned)(w.Rpad / 32), (unsigned)(w.Lp / 32)), 256, 0, st>>>(w.xf, w.Rpad, (int)w.Lp,
                                                                                             w.scl, w.x16, w.xT);
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

inline int rc_sweep(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                    float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
{
    // CLUSCO_BACKWARD_CLUSTERS=0 runs the chunk CTAs without clusters (each recomputes the
    // rotations of every tile): the same results, for comparison and for devices without clusters
    const char *ev = getenv("CLUSCO_BACKWARD_CLUSTERS");
    const bool allow_cluster = !(ev && ev[0] == '0');
    const RcWs w = carve_rc(ws, N, L);
    cudaError_t e = cudaSuccess;
    // tensor maps: x16 [2 Rpad][Lp] (boxes of 64 atoms x 128 or 64 rows), xT parts [Lp][Rpad]
    // (boxes of the tile's 64 rows x 128 atoms; atoms past Lp read as zeros)
    CUtensorMap mXA, mXB, mTh, mTl;
    auto enc = [&](CUtensorMap *m, void *base, uint64_t inner, uint64_t outer, uint32_t bx, uint32_t by) {
        const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
        const cuuint64_t strides[1] = {(cuuint64_t)(inner * 2)};
        const cuuint32_t box[2] = {bx, by};
        const cuuint32_t estr[2] = {1, 1};
        return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    if (enc(&mXA, w.x16, (uint64_t)w.Lp, (uint64_t)(2 * w.Rpad), 64u, 128u) != CUDA_SUCCESS ||
        enc(&mXB, w.x16, (uint64_t)w.Lp, (uint64_t)(2 * w.Rpad), 64u, 64u) != CUDA_SUCCESS ||
        enc(&mTh, w.xT, (uint64_t)w.Rpad, (uint64_t)w.Lp, 64u, (uint32_t)RC_BLK) != CUDA_SUCCESS ||
        enc(&mTl, w.xT + w.Lp * w.Rpad, (uint64_t)w.Rpad, (uint64_t)w.Lp, 64u, (uint32_t)RC_BLK) != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled (backward operands) failed";
        return CLUSCO_ECUDA;
    }
    const int64_t TA = w.Npad / TC_MA, TB = w.Npad / TC_MB;
    const int nkb = (int)(w.Lp / 64);
    e = cudaFuncSetAttribute(bwd_rc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC_SMEM);
    if (e != cudaSuccess) {
        err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return CLUSCO_ECUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(TA * w.C));  // the grid's x is set below, with the column ranges
    cfg.blockDim = dim3(RC_THREADS);
    cfg.dynamicSmemBytes = RC_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)w.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    int CS = 1;
    int64_t resident = 0;  // work groups the device runs at once
    if (w.C > 1 && allow_cluster) {
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, bwd_rc_kernel, &cfg) == cudaSuccess && nclusters > 0) {
            CS = (int)w.C;
            resident = nclusters;
        } else {
            (void)cudaGetLastError();  // clear: fall back to independent chunk CTAs
        }
    }
    if (CS == 1) {
        cfg.attrs = nullptr;
        cfg.numAttrs = 0;
        int dev = 0, sms = 148, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd_rc_kernel, RC_THREADS, RC_SMEM) != cudaSuccess ||
            per_sm < 1) {
            (void)cudaGetLastError();
            per_sm = 1;
        }
        resident = (int64_t)sms * per_sm / w.C;  // a group is C chunk CTAs
    }
    const int64_t S = rc_pick_splits(TA, TB, w.Smax, resident);
    const int64_t JC = (TB + S - 1) / S;
    cfg.gridDim = dim3((unsigned)(TA * S * w.C));
    prof_mark(PROF_ADJOINT, st);
    e = cudaLaunchKernelEx(&cfg, bwd_rc_kernel, mXA, mXB, mTh, mTl, (const float *)w.G32, N, (int)L, (int)w.Lp, nkb,
                           w.Rpad, TB, S, JC, (int)w.C, (int)w.q, (int)w.nblk, CS, crmsd, grad_out, eps,
                           (const unsigned *)w.scl, w.Gp, w.dp, w.nd_list, w.nd_count, w.nd_cap);
    prof_mark(PROF_ADJOINT, st);
    if (e == cudaSuccess) {
        if (w.Lp <= 128 * BRED_MAXQ)
            bwd_reduce_kernel<BRED_MAXQ><<<(unsigned)N, BRED_THREADS, (size_t)(3 * L * sizeof(float)), st>>>(
                w.Gp, w.dp, w.xf, N, (int)L, (int)w.Lp, w.Rpad, S, S * w.C, grad);
        else
            bwd_reduce_kernel<8><<<(unsigned)N, BRED_THREADS, (size_t)(3 * L * sizeof(float)), st>>>(
                w.Gp, w.dp, w.xf, N, (int)L, (int)w.Lp, w.Rpad, S, S * w.C, grad);
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

inline int rc_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                     float *grad, float eps, void *ws, cudaStream_t st, std::string &err)
{
    const int rc = rc_prepare(coords, N, L, grad_out, ws, st, err);
    return rc ? rc : rc_sweep(coords, N, L, grad_out, crmsd, grad, eps, ws, st, err);
}

inline size_t backward_ws_bytes(int64_t N, int64_t L, int form)
{
    (void)form;
    size_t a = backward_simt_ws_bytes(N, L);
    if (rc_supported(L)) {
        const size_t b = carve_rc(nullptr, N, L).bytes;
        if (b > a) a = b;
    }
    return a;
}

// The adjoint: the tensor-core path (rotations recomputed, clusters sharing them) when the device
// and L allow it, else the CUDA-core path.
inline int backward_launch(const float *coords, int64_t N, int64_t L, const float *grad_out, const float *crmsd,
                           float *grad, float eps, int form, void *ws, cudaStream_t st, std::string &err)
{
    if (rc_supported(L) && tc_supported(CLUSCO_FORM_BF16_EXACT2, L) == CLUSCO_OK)
        return rc_launch(coords, N, L, grad_out, crmsd, grad, eps, ws, st, err);
    return backward_simt_launch(coords, N, L, grad_out, crmsd, grad, eps, form, ws, st, err);
}

}  // namespace clusco

// epilogue.cuh -- per-pair cRMSD from a 3x3 covariance (eq. 2), FP32 and FP64 forms.
//
// For centred models A, B with H = sum_i a_i b_i^T and G_A = sum_i |a_i|^2,
// G_B = sum_i |b_i|^2, eq. 2 reads
//     L * cRMSD^2 = G_A + G_B - 2 (s1 + s2 + S s3)
// with s_k the singular values of H (square roots of the eigenvalues of
// H^T H, the roots of its characteristic cubic) and S = sign(det H).
//
// Everything here works in a normalised frame m = H * 2 / (G_A + G_B), so that
// Sigma_hat = s1 + s2 + S s3 of m lies in [-1, 1] and
//     L * cRMSD^2 = (G_A + G_B) (1 - Sigma_hat);
// no intermediate can overflow whatever the coordinate scale, and the
// cancellation sits in one subtraction 1 - Sigma_hat.
//
// Two refinements of Sigma_hat are used beside the cubic:
//   Sigma = s1 + s2 + S s3 is the largest root of the quartic
//     P(x) = x^4 - 2 I1 x^2 - 8 det(m) x + (I1^2 - 4 I2),
//   I1 = |m|_F^2, I2 = sum of squared 2x2 minors of m (= e2 of m^T m by
//   Cauchy-Binet); its roots are +-s1 +- s2 +- s3 with sign product S. P is
//   convex right of its largest root, so Newton steps from the cubic's
//   estimate converge to it quadratically.
#pragma once
#include <cuda_runtime.h>


// Paired FP32 arithmetic: two IEEE operations (round to nearest) per instruction on the halves
// of a float2, so that one lane carries two independent pairs.
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&d);
}
// a b - c d
__device__ __forceinline__ float2 dif2(float2 a, float2 b, float2 c, float2 d) { return sub2(mul2(a, b), mul2(c, d)); }

// The nine 2x2 minors of m (row-major), mn = {a01, a02, a12, b01, b02, b12, c01, c02, c12}:
// a.. from rows 1,2, b.. from rows 0,2, c.. from rows 0,1; the digits name the columns.
template <typename T>
__device__ __forceinline__ void minors3(const T m[9], T mn[9])
{
    mn[0] = m[3] * m[7] - m[4] * m[6];
    mn[1] = m[3] * m[8] - m[5] * m[6];
    mn[2] = m[4] * m[8] - m[5] * m[7];
    mn[3] = m[0] * m[7] - m[1] * m[6];
    mn[4] = m[0] * m[8] - m[2] * m[6];
    mn[5] = m[1] * m[8] - m[2] * m[7];
    mn[6] = m[0] * m[4] - m[1] * m[3];
    mn[7] = m[0] * m[5] - m[2] * m[3];
    mn[8] = m[1] * m[5] - m[2] * m[4];
}

// Invariants of the 3x3 matrix m from its minors: I1 = |m|^2, det, I2 = sum of squared minors.
template <typename T>
__device__ __forceinline__ void invariants_from_minors(const T m[9], const T mn[9], T &I1, T &det, T &I2)
{
    det = m[0] * mn[2] - m[1] * mn[1] + m[2] * mn[0];
    I2 = mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2] + mn[3] * mn[3] + mn[4] * mn[4] + mn[5] * mn[5]
       + mn[6] * mn[6] + mn[7] * mn[7] + mn[8] * mn[8];
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) s += m[k] * m[k];
    I1 = s;
}

// Invariants of the 3x3 matrix m (row-major): I1 = |m|^2, det, I2 = sum of squared 2x2 minors.
template <typename T>
__device__ __forceinline__ void invariants3(const T m[9], T &I1, T &det, T &I2)
{
    T mn[9];
    minors3(m, mn);
    invariants_from_minors(m, mn, I1, det, I2);
}

// Eq. 2's route: the eigenvalues l1 >= l2 >= l3 of m^T m are the roots of
//   l^3 - I1 l^2 + I2 l - det^2 = 0.
// The largest root l1 comes from the trigonometric (Viete) solution, where it is well
// conditioned. The other two enter only through sqrt(l2) + S sqrt(l3), whose square is
//   l2 + l3 + 2 S sqrt(l2 l3) = (I2 - det^2/l1)/l1 + 2 det/sqrt(l1)
// by Vieta's relations (l2 + l3 = (I2 - l2 l3)/l1, l2 l3 = det^2/l1, S |det| = det).
// I2 is a sum of squared 2x2 minors, so a rank-deficient m (collinear or planar atoms)
// keeps full relative accuracy, which sqrt() of the small cubic roots would lose.
// Returns Sigma = sqrt(l1) + sqrt(l2) + S sqrt(l3). FP64, IEEE operations.
__device__ __forceinline__ double sigma_cubic_d(double I1, double det, double I2)
{
    const double mm = I1 / 3.0;
    const double p = I2 - 3.0 * mm * mm;  // <= 0 for a real symmetric spectrum
    const double q = (I2 - 2.0 * mm * mm) * mm - det * det;
    double l1;
    if (!(p < 0.0)) {
        l1 = mm;
    } else {
        const double r = sqrt(-p / 3.0);
        double arg = (3.0 * q / (2.0 * p)) * sqrt(-3.0 / p);
        arg = fmin(fmax(arg, -1.0), 1.0);
        l1 = mm + 2.0 * r * cos(acos(arg) / 3.0);
    }
    if (!(l1 > 0.0)) return 0.0;
    const double rl1 = sqrt(l1);
    const double t = (I2 - det * det / l1) / l1 + 2.0 * det / rl1;
    return rl1 + sqrt(fmax(t, 0.0));
}

// The same in FP32 with hardware approximations (reciprocal, reciprocal square root,
// cosine): a starting value for the FP32 Newton polish, accurate to about 1e-6.
__device__ __forceinline__ float sigma_cubic_f(float I1, float det, float I2)
{
    // branch-free (selects), so that independent pairs interleave
    const float mm = I1 * (1.f / 3.f);
    const float p = I2 - 3.f * mm * mm;
    const float q = (I2 - 2.f * mm * mm) * mm - det * det;
    const float pn = fminf(p, -1e-30f);
    const float rp = rsqrtf(-pn);               // 1/sqrt(-p)
    const float r = -pn * rp * 0.57735026919f;  // sqrt(-p/3)
    float arg = 1.5f * q * __fdividef(1.f, pn) * 1.73205080757f * rp;  // (3q/2p) sqrt(-3/p)
    arg = fminf(fmaxf(arg, -1.f), 1.f);
    float l1 = fmaf(2.f * r, __cosf(acosf(arg) * (1.f / 3.f)), mm);
    l1 = (p < 0.f) ? l1 : mm;
    const bool pos = l1 > 0.f;
    const float l1p = pos ? l1 : 1.f;
    const float rl1i = rsqrtf(l1p);
    const float il1 = rl1i * rl1i;
    const float t = fmaxf((I2 - det * det * il1) * il1 + 2.f * det * rl1i, 0.f);
    const float st = (t > 0.f) ? t * rsqrtf(t) : 0.f;  // a start value: approximate sqrt is enough
    return pos ? l1p * rl1i + st : 0.f;
}

// Newton steps on the quartic whose largest root is s1 + s2 + S s3. At that root
// P' = 8 (s2 + S s3)(s1 + S s3)(s1 + s2); where it vanishes against 8 Sigma^3 (rank <= 1
// covariance, or S = -1 with s2 = s3) the root is double, P and P' are rounding noise and
// a Newton step would be noise over noise, so no step is taken once P' falls below 1e-3
// of its natural scale and *degenerate is set; the cubic route is the answer there.
template <typename T>
__device__ __forceinline__ T quartic_newton(T s, T I1, T det, T I2, int iters, bool *degenerate)
{
    const T c2 = T(-2) * I1;
    const T c1 = T(-8) * det;
    const T c0 = I1 * I1 - T(4) * I2;
    bool deg = false;
    for (int it = 0; it < iters; ++it) {
        const T s2 = s * s;
        const T P = (s2 + c2) * s2 + c1 * s + c0;
        const T dP = (T(4) * s2 + T(2) * c2) * s + c1;
        if (dP > T(8e-3) * s2 * s) {
            s -= P / dP;
        } else {
            deg = true;
        }
    }
    *degenerate = deg;
    return s;
}

__device__ __forceinline__ float quartic_newton_f(float s, float I1, float det, float I2, int iters, bool *degenerate,
                                                  float *dP_out)
{
    const float c2 = -2.f * I1;
    const float c1 = -8.f * det;
    const float c0 = I1 * I1 - 4.f * I2;
    bool deg = false;
    float dP = 0.f;
#pragma unroll
    for (int it = 0; it < iters; ++it) {
        const float s2 = s * s;
        const float P = fmaf(s2 + c2, s2, fmaf(c1, s, c0));
        dP = fmaf(fmaf(4.f, s2, 2.f * c2), s, c1);
        if (dP > 8e-3f * s2 * s) {
            s -= __fdividef(P, dP);
        } else {
            deg = true;
        }
    }
    *degenerate = deg;
    *dP_out = dP;
    return s;
}

// The plain form's epilogue, FP64 throughout: the cubic route only, no Newton polish.
// H is the raw covariance, Ga/Gb the raw sums of squares, invL = 1/L.
__device__ __forceinline__ float crmsd_plain_fp64(const double H[9], double Ga, double Gb, double invL)
{
    const double Gs = Ga + Gb;
    if (!(Gs > 0.0)) return 0.0f;
    const double nrm = 2.0 / Gs;
    double m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = H[k] * nrm;
    double I1, det, I2;
    invariants3(m, I1, det, I2);
    const double s = sigma_cubic_d(I1, det, I2);
    const double c2 = Gs * invL * (1.0 - s);
    return (float)sqrt(fmax(c2, 0.0));
}

// FP64 refinement: exact covariance in; start from s_start (an FP32 estimate) when given,
// Newton polish; a degenerate (double) root falls back to the FP64 cubic route.
// The cancellation 1 - Sigma_hat is taken in FP64. Returns cRMSD.
__device__ __forceinline__ double crmsd_refined_fp64(const double H[9], double Ga, double Gb, double invL,
                                                     double s_start, bool have_start)
{
    const double Gs = Ga + Gb;
    if (!(Gs > 0.0)) return 0.0;
    const double nrm = 2.0 / Gs;
    double m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = H[k] * nrm;
    double I1, det, I2;
    invariants3(m, I1, det, I2);
    double s = have_start ? s_start : sigma_cubic_d(I1, det, I2);
    bool deg;
    s = quartic_newton(s, I1, det, I2, 3, &deg);
    if (deg) s = sigma_cubic_d(I1, det, I2);
    const double c2 = Gs * invL * (1.0 - s);
    return sqrt(fmax(c2, 0.0));
}

// FP64 refinement of a pair the FP32 fast path flagged, from its exact covariance H (raw
// units) and the fast path's estimate s_hat of Sigma_hat = 2 Sigma / (G_A + G_B).
// m = H 2^-e with 2^e <= G_A + G_B < 2^(e+1): a power of two, so the normalisation is exact
// and needs no division. Newton steps on the quartic take the correction P / P' with an
// FP32 reciprocal of P': its relative error (2^-24) scales only the correction, so the
// iteration still converges to the FP64 root (from an FP32 start, one step reaches about
// 1e-14). A degenerate root (P' below 8e-3 s^3) takes the FP64 cubic route instead.
// c^2 = (G_A + G_B - 2 Sigma) / L = 2^(e+1) (h - s) / L with h = (G_A + G_B) 2^-e / 2, the
// cancellation taken in FP64. invL is 1/L in FP64. Returns cRMSD rounded to FP32.
__device__ __forceinline__ float crmsd_refine_newton_fp64(const double H[9], double Ga, double Gb, double invL,
                                                          float s_hat)
{
    const double Gs = Ga + Gb;
    if (!(Gs > 1e-300)) return 0.f;  // c^2 <= Gs / L: zero in FP32
    if (!(Gs < 1.7e308)) return __int_as_float(0x7fc00000);
    const long long ebits = (__double_as_longlong(Gs) >> 52) & 0x7ff;  // biased exponent, 1..2046
    const double p2 = __longlong_as_double((2046LL - ebits) << 52);     // 2^-e
    const double ip2 = __longlong_as_double(ebits << 52);                // 2^e
    double m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = H[k] * p2;
    double I1, det, I2;
    invariants3(m, I1, det, I2);
    const double h = 0.5 * (Gs * p2);  // in [0.5, 1)
    const double c2c = -2.0 * I1, c1 = -8.0 * det, c0 = I1 * I1 - 4.0 * I2;
    double s = (double)s_hat * h;
    bool deg = false;
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        const double s2 = s * s;
        const double P = (s2 + c2c) * s2 + c1 * s + c0;
        const double dP = (4.0 * s2 + 2.0 * c2c) * s + c1;
        if (dP > fmax(8e-3 * s2 * s, 1e-30))
            s -= P * (double)__frcp_rn((float)dP);
        else
            deg = true;
    }
    if (deg) s = sigma_cubic_d(I1, det, I2);
    const double c2 = 2.0 * (h - s) * ip2 * invL;
    return sqrtf((float)fmax(c2, 0.0));
}

// Sigma_hat alone (FP32, cubic start + two Newton steps) for a normalised covariance m:
// what the adjoint needs for the rotation, without cRMSD or its error bound.
__device__ __forceinline__ float sigma_hat_f32(const float m[9])
{
    float I1, det, I2, dP;
    bool deg;
    invariants3(m, I1, det, I2);
    return quartic_newton_f(sigma_cubic_f(I1, det, I2), I1, det, I2, 2, &deg, &dP);
}

// Sigma and the optimal rotation together, FP32, for a normalised covariance m (row-major).
// The rotation maximises <R, m> over SO(3) with maximum Sigma, so by the envelope theorem it
// is dSigma/dm; Sigma is the largest root of P(x; I1, I2, det) = 0 (the quartic above), and
// implicit differentiation with dI1/dm = 2 m, dI2/dm = 2 I1 m - 2 m m^T m, ddet/dm = cof(m)
// gives
//   R = [4 (I1 + Sigma^2) m - 8 m m^T m + 8 Sigma cof(m)] / P'(Sigma),
//   P'(Sigma) = 4 Sigma^3 - 4 I1 Sigma - 8 det.
// The cofactors are the 2x2 minors that I2 and det are built from. rotation_from_sigma_f32
// takes Sigma (of m) as computed; both return false, leaving R unset, where P' falls below
// 1e-2 of 8 Sigma^3 (near a double root, where this quotient loses accuracy); the caller then
// takes the eigenvector route of rotation.cuh.
__device__ __forceinline__ float2 f2b(float x) { return make_float2(x, x); }

// The rotation from m, its minors mn (minors3), det, I1 and Sigma s. Columns 0 and 1 of every
// 3 x 3 product go through the paired FP32 instructions (__ffma2_rn: two IEEE FMAs per
// instruction), column 2 through scalar FMAs.
__device__ __forceinline__ bool rotation_core_f32(const float m[9], const float mn[9], float det, float I1, float s,
                                                  float R[9])
{
    const float s2 = s * s;
    const float dP = fmaf(fmaf(4.f, s2, -4.f * I1), s, -8.f * det);
    if (!(dP > 8e-2f * s2 * s)) return false;
    // cofactor matrix (signed minors), row-major: columns 0, 1 as pairs, column 2 alone
    const float2 cf01[3] = {make_float2(mn[2], -mn[1]), make_float2(-mn[5], mn[4]), make_float2(mn[8], -mn[7])};
    const float cf2[3] = {mn[0], -mn[3], mn[6]};
    float2 v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = make_float2(m[3 * i], m[3 * i + 1]);
    // g = m^T m (symmetric): (g00, g11), (g02, g12) as pairs
    float2 gd = __fmul2_rn(v[0], v[0]);
    gd = __ffma2_rn(v[1], v[1], gd);
    gd = __ffma2_rn(v[2], v[2], gd);
    float2 gc = __fmul2_rn(v[0], f2b(m[2]));
    gc = __ffma2_rn(v[1], f2b(m[5]), gc);
    gc = __ffma2_rn(v[2], f2b(m[8]), gc);
    const float g01 = fmaf(m[6], m[7], fmaf(m[3], m[4], m[0] * m[1]));
    const float g22 = fmaf(m[8], m[8], fmaf(m[5], m[5], m[2] * m[2]));
    const float2 gA = make_float2(gd.x, g01), gB = make_float2(g01, gd.y);
    const float inv = __fdividef(1.f, dP);
    const float al = 4.f * (I1 + s2) * inv, be = 8.f * s * inv, ga = -8.f * inv;
    float2 R01[3];
    float R2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float r0 = m[3 * i], r1 = m[3 * i + 1], r2 = m[3 * i + 2];
        float2 mg = __fmul2_rn(f2b(r0), gA);
        mg = __ffma2_rn(f2b(r1), gB, mg);
        mg = __ffma2_rn(f2b(r2), gc, mg);
        const float mg2 = fmaf(r2, g22, fmaf(r1, gc.y, r0 * gc.x));
        float2 t = __fmul2_rn(f2b(be), cf01[i]);
        t = __ffma2_rn(f2b(ga), mg, t);
        R01[i] = __ffma2_rn(f2b(al), v[i], t);
        R2[i] = fmaf(al, r2, fmaf(ga, mg2, be * cf2[i]));
    }
    // The quotient inherits Sigma's FP32 error amplified by about Q/P', mostly as a departure
    // from orthogonality; one Newton-Schulz step R <- R (3 I - R^T R) / 2 removes that to
    // second order (the polar factor of R is the nearest rotation). q = R^T R with (q00, q11),
    // (q02, q12) as pairs.
    float2 qd = __fmul2_rn(R01[0], R01[0]);
    qd = __ffma2_rn(R01[1], R01[1], qd);
    qd = __ffma2_rn(R01[2], R01[2], qd);
    float2 qc = __fmul2_rn(R01[0], f2b(R2[0]));
    qc = __ffma2_rn(R01[1], f2b(R2[1]), qc);
    qc = __ffma2_rn(R01[2], f2b(R2[2]), qc);
    const float q01 = fmaf(R01[2].x, R01[2].y, fmaf(R01[1].x, R01[1].y, R01[0].x * R01[0].y));
    const float q22 = fmaf(R2[2], R2[2], fmaf(R2[1], R2[1], R2[0] * R2[0]));
    const float2 td = __ffma2_rn(f2b(-0.5f), qd, f2b(1.5f));  // (t00, t11)
    const float2 tc = __fmul2_rn(f2b(-0.5f), qc);             // (t02, t12)
    const float t01 = -0.5f * q01, t22 = fmaf(-0.5f, q22, 1.5f);
    const float2 tA = make_float2(td.x, t01), tB = make_float2(t01, td.y);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float r0 = R01[i].x, r1 = R01[i].y, r2 = R2[i];
        float2 o = __fmul2_rn(f2b(r0), tA);
        o = __ffma2_rn(f2b(r1), tB, o);
        o = __ffma2_rn(f2b(r2), tc, o);
        R[3 * i + 0] = o.x;
        R[3 * i + 1] = o.y;
        R[3 * i + 2] = fmaf(r2, t22, fmaf(r1, tc.y, r0 * tc.x));
    }
    return true;
}

__device__ __forceinline__ bool rotation_from_sigma_f32(const float m[9], float s, float R[9])
{
    float mn[9];
    minors3(m, mn);
    const float det = m[0] * mn[2] - m[1] * mn[1] + m[2] * mn[0];
    float I1 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) I1 = fmaf(m[k], m[k], I1);
    return rotation_core_f32(m, mn, det, I1, s, R);
}

__device__ __forceinline__ bool sigma_rotation_f32(const float m[9], float R[9])
{
    return rotation_from_sigma_f32(m, sigma_hat_f32(m), R);
}

// Sigma and the rotation from one set of minors, starting the Newton steps from a known
// estimate s0 of Sigma_hat instead of the cubic: the recomputing adjoint has the forward's
// cRMSD c of the pair, and L c^2 = (G_A + G_B)(1 - Sigma_hat), so s0 = 1 - L c^2 / (G_A + G_B)
// is within the forward's error of the root; one Newton step on this covariance's own quartic
// (quadratic convergence) takes it to the root of the matrix at hand. False, R unset, where the
// closed form is ill-conditioned (see rotation_core_f32).
__device__ __forceinline__ bool sigma_rotation_from_f32(const float m[9], float s0, float R[9])
{
    float mn[9];
    minors3(m, mn);
    float I1, det, I2, dP;
    invariants_from_minors(m, mn, I1, det, I2);
    bool deg;
    const float s = quartic_newton_f(s0, I1, det, I2, 1, &deg, &dP);
    return rotation_core_f32(m, mn, det, I1, s, R);
}

// Sigma and the rotation from one set of minors (I1, I2 and det for the cubic and the Newton
// steps, the cofactors for the rotation): the recomputing adjoint's per-pair work. False, R
// unset, where the closed form is ill-conditioned (see rotation_core_f32).
__device__ __forceinline__ bool sigma_rotation_once_f32(const float m[9], float R[9])
{
    float mn[9];
    minors3(m, mn);
    float I1, det, I2, dP;
    invariants_from_minors(m, mn, I1, det, I2);
    bool deg;
    const float s = quartic_newton_f(sigma_cubic_f(I1, det, I2), I1, det, I2, 2, &deg, &dP);
    return rotation_core_f32(m, mn, det, I1, s, R);
}

// FP32 fast path on a rounded covariance: cubic start + two Newton steps, all FP32.
// Returns cRMSD and, through err_c2, a bound on the absolute error of cRMSD^2 from FP32
// rounding. The bound follows the root's conditioning: the quartic is evaluated with an
// error of a few ulps of Q = s^4 + 2 I1 s^2 + 8 |det| s + I1^2 (its terms' magnitudes),
// which moves the root by that over P'(s); measured on 2e8 pairs of the precision and
// bench ensembles, |d(c^2)| / (ulp * (G_A+G_B)/L) never exceeded 6 + 0.6 Q/P', and the
// bound uses KERR_A + KERR_B Q/P' with KERR_A = 8, KERR_B = 1. The worst cases are S = -1
// with s2 ~ s3 (a near-double root). A degenerate root returns err_c2 = +inf so that the
// caller refines the pair.
#ifndef CLUSCO_KERR_A
#define CLUSCO_KERR_A 8.0f
#endif
#ifndef CLUSCO_KERR_B
#define CLUSCO_KERR_B 1.0f
#endif
__device__ __forceinline__ float crmsd_fast_fp32(const float H[9], float Ga, float Gb, float invL, float *s_out,
                                                 float *err_c2)
{
    const float Gs = Ga + Gb;
    const bool pos = Gs > 0.0f;
    const float nrm = __fdividef(2.0f, pos ? Gs : 1.0f);
    float m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = H[k] * nrm;
    float I1, det, I2;
    invariants3(m, I1, det, I2);
    bool deg;
    float dP;
    const float s = quartic_newton_f(sigma_cubic_f(I1, det, I2), I1, det, I2, 2, &deg, &dP);
    *s_out = s;
    const float scale = Gs * invL;
    const float s2 = s * s;
    const float Q = fmaf(s2 + 2.f * I1, s2, fmaf(8.f * fabsf(det), s, I1 * I1));
    const float kq = CLUSCO_KERR_A + CLUSCO_KERR_B * __fdividef(Q, dP);
    const float e = (deg || !(dP > 0.f)) ? __int_as_float(0x7f800000) : kq * 5.9604645e-8f * scale;
    *err_c2 = pos ? e : 0.0f;
    return pos ? sqrtf(fmaxf(scale * (1.0f - s), 0.0f)) : 0.0f;
}

// crmsd_fast_fp32 for two pairs at once, one in each half of a float2: the same steps on the
// paired FP32 instructions, the cubic's start, the reciprocals and the square root per pair.
__device__ __forceinline__ float2 crmsd_fast_fp32x2(const float2 H[9], float2 Ga, float2 Gb, float invL,
                                                   float2 *err_c2)
{
    const float2 Gs = add2(Ga, Gb);
    const bool posx = Gs.x > 0.0f, posy = Gs.y > 0.0f;
    const float2 nrm = make_float2(__fdividef(2.0f, posx ? Gs.x : 1.0f), __fdividef(2.0f, posy ? Gs.y : 1.0f));
    float2 m[9], mn[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = mul2(H[k], nrm);
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
    // the cubic's start per pair, then two Newton steps on the quartic (see quartic_newton_f)
    float2 s = make_float2(sigma_cubic_f(I1.x, det.x, I2.x), sigma_cubic_f(I1.y, det.y, I2.y));
    const float2 c2 = mul2(bc2(-2.f), I1), c1 = mul2(bc2(-8.f), det);
    const float2 c0 = fma2(I1, I1, mul2(bc2(-4.f), I2));
    float2 dP = bc2(0.f);
    bool degx = false, degy = false;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const float2 sq = mul2(s, s);
        const float2 P = fma2(add2(sq, c2), sq, fma2(c1, s, c0));
        dP = fma2(fma2(bc2(4.f), sq, mul2(bc2(2.f), c2)), s, c1);
        const float2 lim = mul2(mul2(bc2(8e-3f), sq), s);
        if (dP.x > lim.x)
            s.x -= __fdividef(P.x, dP.x);
        else
            degx = true;
        if (dP.y > lim.y)
            s.y -= __fdividef(P.y, dP.y);
        else
            degy = true;
    }
    // the error bound of crmsd_fast_fp32
    const float2 scale = mul2(Gs, bc2(invL));
    const float2 sq = mul2(s, s);
    const float2 adet = make_float2(fabsf(det.x), fabsf(det.y));
    const float2 Q = fma2(fma2(bc2(2.f), I1, sq), sq, fma2(mul2(bc2(8.f), adet), s, mul2(I1, I1)));
    const float2 kq = make_float2(CLUSCO_KERR_A + CLUSCO_KERR_B * __fdividef(Q.x, dP.x),
                                  CLUSCO_KERR_A + CLUSCO_KERR_B * __fdividef(Q.y, dP.y));
    const float2 e = mul2(mul2(kq, bc2(5.9604645e-8f)), scale);
    err_c2->x = posx ? ((degx || !(dP.x > 0.f)) ? __int_as_float(0x7f800000) : e.x) : 0.0f;
    err_c2->y = posy ? ((degy || !(dP.y > 0.f)) ? __int_as_float(0x7f800000) : e.y) : 0.0f;
    const float2 d = fma2(scale, sub2(bc2(0.f), s), scale);  // scale (1 - s)
    return make_float2(posx ? sqrtf(fmaxf(d.x, 0.0f)) : 0.0f, posy ? sqrtf(fmaxf(d.y, 0.0f)) : 0.0f);
}

// crmsd_fast_fp32 and the rotation of the same pair together: one set of minors serves I2,
// det and the rotation's cofactor term. m receives the normalised block (the rotation's
// input, for callers that defer the rare pairs whose quotient is ill-conditioned: *okR false).
__device__ __forceinline__ float crmsd_fast_rot_fp32(const float H[9], float Ga, float Gb, float invL, float *s_out,
                                                     float *err_c2, float m[9], float R[9], bool *okR)
{
    const float Gs = Ga + Gb;
    const bool pos = Gs > 0.0f;
    const float nrm = __fdividef(2.0f, pos ? Gs : 1.0f);
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = H[k] * nrm;
    float mn[9];
    minors3(m, mn);
    float I1, det, I2;
    invariants_from_minors(m, mn, I1, det, I2);
    bool deg;
    float dP;
    const float s = quartic_newton_f(sigma_cubic_f(I1, det, I2), I1, det, I2, 2, &deg, &dP);
    *s_out = s;
    const float scale = Gs * invL;
    const float s2 = s * s;
    const float Q = fmaf(s2 + 2.f * I1, s2, fmaf(8.f * fabsf(det), s, I1 * I1));
    const float kq = CLUSCO_KERR_A + CLUSCO_KERR_B * __fdividef(Q, dP);
    const float e = (deg || !(dP > 0.f)) ? __int_as_float(0x7f800000) : kq * 5.9604645e-8f * scale;
    *err_c2 = pos ? e : 0.0f;
    *okR = rotation_core_f32(m, mn, det, I1, s, R);
    return pos ? sqrtf(fmaxf(scale * (1.0f - s), 0.0f)) : 0.0f;
}

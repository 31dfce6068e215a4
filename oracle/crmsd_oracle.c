/*
 * crmsd_oracle.c -- FP64 CPU oracle for all-versus-all cRMSD.
 *
 * TEST INFRASTRUCTURE. This is the plain, slow, obviously-correct reference
 * that the CUDA path is checked against. Only the tests, the smoke check and
 * the bench's CPU-baseline leg may load it. It shares no code, header, helper
 * or constant with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (ClusCo, section "Algorithms", eq. 1 with the cited
 * Kabsch superposition):
 *
 *   cRMSD(A, B) = min over proper rotations R and translations t of
 *                 sqrt( (1/L) * sum_i |a_i - R b_i - t|^2 )
 *
 * over L matched atoms. Steps, in this order, all in FP64 (the FP32 input
 * coordinates are promoted exactly):
 *   1. centre each model on its centroid (the optimal t is the centroid
 *      difference);
 *   2. H = sum_i a_i b_i^T over the centred coordinates (3x3);
 *   3. one-sided Jacobi SVD H = U diag(s) V^T, swept until every column pair
 *      is orthogonal to 4 ulp or one of the two is numerically zero (at most
 *      64 sweeps, failure reported);
 *   4. the optimal proper rotation R = U diag(1, 1, d) V^T with
 *      d = sign(det(U V^T)) (Kabsch);
 *   5. the RMS of the residuals a_i - R b_i, computed directly from the
 *      residuals so that there is no cancellation as cRMSD -> 0.
 *
 * The gradient of the weighted loss sum_{a<b} w_ab cRMSD_ab follows from the
 * envelope theorem (R and t optimal): d cRMSD / d a_i = (a_i - R b_i)/(L c),
 * the chain rule through the centring, and the guarded denominator
 * L * max(c, eps) (the guard reading: the denominator is clamped, the
 * residual is not).
 *
 * oracle_crmsd_eq2 restates the paper's own closed form (eq. 2): the
 * eigenvalues of M^T M as the roots of a cubic (trigonometric solution),
 * S = sign(det M), cRMSD = sqrt(R_A^2 + R_B^2 - 2 (sqrt l1 + sqrt l2 + S sqrt l3)).
 * It is a second CPU method, used as a pin against the Kabsch path and as an
 * optional CPU baseline; the oracle's answers never come from it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOCONV 2

/* ---- step 1: centring ------------------------------------------------- */
static void centre(const float *x, int64_t L, double *xc)
{
    double m[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < L; ++i)
        for (int k = 0; k < 3; ++k) m[k] += (double)x[3 * i + k];
    for (int k = 0; k < 3; ++k) m[k] /= (double)L;
    for (int64_t i = 0; i < L; ++i)
        for (int k = 0; k < 3; ++k) xc[3 * i + k] = (double)x[3 * i + k] - m[k];
}

/* ---- step 2: covariance H = sum_i a_i b_i^T ---------------------------- */
static void covariance(const double *ac, const double *bc, int64_t L, double H[3][3])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) H[r][c] = 0.0;
    for (int64_t i = 0; i < L; ++i)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) H[r][c] += ac[3 * i + r] * bc[3 * i + c];
}

static double det3(const double A[3][3])
{
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* ---- step 3: one-sided Jacobi SVD of a 3x3 matrix ---------------------- */
/* Returns 0 on convergence. On return H = U diag(s) V^T with s descending,
 * U and V orthogonal. */
static int svd3(const double H[3][3], double U[3][3], double s[3], double V[3][3])
{
    double W[3][3];
    memcpy(W, H, sizeof W);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V[r][c] = (r == c) ? 1.0 : 0.0;

    const double tol = 4.0 * 2.220446049250313e-16;
    /* a column whose squared norm is below (tol |H|)^2 is numerically zero: its singular value
     * is 0 and its direction is completed below, so it takes no rotation (without this floor a
     * rank-deficient H, e.g. three reference atoms in one coordinate plane, can cycle forever) */
    double hn2 = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) hn2 += H[r][c] * H[r][c];
    const double zero_col = tol * tol * hn2;
    int converged = 0;
    for (int sweep = 0; sweep < 64 && !converged; ++sweep) {
        converged = 1;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < 3; ++i) {
                    alpha += W[i][p] * W[i][p];
                    beta += W[i][q] * W[i][q];
                    gamma += W[i][p] * W[i][q];
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta) || alpha <= zero_col || beta <= zero_col)
                    continue;
                converged = 0;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (int i = 0; i < 3; ++i) {
                    double wp = W[i][p], wq = W[i][q];
                    W[i][p] = c * wp - sn * wq;
                    W[i][q] = sn * wp + c * wq;
                    double vp = V[i][p], vq = V[i][q];
                    V[i][p] = c * vp - sn * vq;
                    V[i][q] = sn * vp + c * vq;
                }
            }
        }
    }
    if (!converged) return ORACLE_ENOCONV;

    /* singular values = column norms; sort descending (columns of W and V) */
    int idx[3] = {0, 1, 2};
    double nrm[3];
    for (int j = 0; j < 3; ++j)
        nrm[j] = sqrt(W[0][j] * W[0][j] + W[1][j] * W[1][j] + W[2][j] * W[2][j]);
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (nrm[idx[b]] > nrm[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    double Vs[3][3];
    for (int j = 0; j < 3; ++j) {
        s[j] = nrm[idx[j]];
        for (int i = 0; i < 3; ++i) { U[i][j] = W[i][idx[j]]; Vs[i][j] = V[i][idx[j]]; }
    }
    memcpy(V, Vs, sizeof Vs);

    /* U columns: W_j / s_j; complete the basis where s_j is (numerically) zero */
    const double rank_tol = 1e-10;
    if (s[0] > 0.0) {
        for (int i = 0; i < 3; ++i) U[i][0] /= s[0];
    } else {
        U[0][0] = 1.0; U[1][0] = 0.0; U[2][0] = 0.0;
    }
    if (s[1] > rank_tol * s[0] && s[0] > 0.0) {
        for (int i = 0; i < 3; ++i) U[i][1] /= s[1];
    } else {
        /* any unit vector orthogonal to U0 */
        double e[3] = {0.0, 0.0, 0.0};
        int k = 0;
        for (int i = 1; i < 3; ++i) if (fabs(U[i][0]) < fabs(U[k][0])) k = i;
        e[k] = 1.0;
        double d = e[0] * U[0][0] + e[1] * U[1][0] + e[2] * U[2][0];
        for (int i = 0; i < 3; ++i) U[i][1] = e[i] - d * U[i][0];
    }
    /* re-orthonormalise U1 against U0 (Gram-Schmidt) */
    {
        double d = U[0][0] * U[0][1] + U[1][0] * U[1][1] + U[2][0] * U[2][1];
        for (int i = 0; i < 3; ++i) U[i][1] -= d * U[i][0];
        double n = sqrt(U[0][1] * U[0][1] + U[1][1] * U[1][1] + U[2][1] * U[2][1]);
        for (int i = 0; i < 3; ++i) U[i][1] /= n;
    }
    if (s[2] > rank_tol * s[0] && s[0] > 0.0) {
        for (int i = 0; i < 3; ++i) U[i][2] /= s[2];
    } else {
        U[0][2] = U[1][0] * U[2][1] - U[2][0] * U[1][1];
        U[1][2] = U[2][0] * U[0][1] - U[0][0] * U[2][1];
        U[2][2] = U[0][0] * U[1][1] - U[1][0] * U[0][1];
    }
    return ORACLE_OK;
}

/* ---- step 4: Kabsch rotation R minimising sum |a_i - R b_i|^2 ----------- */
static int kabsch(const double *ac, const double *bc, int64_t L, double R[3][3])
{
    double H[3][3], U[3][3], V[3][3], s[3];
    covariance(ac, bc, L, H);
    int st = svd3(H, U, s, V);
    if (st) return st;
    double d = (det3(U) * det3(V) < 0.0) ? -1.0 : 1.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[r][c] = U[r][0] * V[c][0] + U[r][1] * V[c][1] + d * U[r][2] * V[c][2];
    return ORACLE_OK;
}

/* ---- step 5: direct RMS of the residuals a_i - R b_i -------------------- */
static double rms_residual(const double *ac, const double *bc, int64_t L, const double R[3][3])
{
    double acc = 0.0;
    for (int64_t i = 0; i < L; ++i) {
        for (int r = 0; r < 3; ++r) {
            double rb = R[r][0] * bc[3 * i + 0] + R[r][1] * bc[3 * i + 1] + R[r][2] * bc[3 * i + 2];
            double e = ac[3 * i + r] - rb;
            acc += e * e;
        }
    }
    return sqrt(acc / (double)L);
}

static int pair_from_centred(const double *ac, const double *bc, int64_t L, double *c, double R[3][3])
{
    int st = kabsch(ac, bc, L, R);
    if (st) return st;
    *c = rms_residual(ac, bc, L, R);
    return ORACLE_OK;
}

static int64_t condensed(int64_t a, int64_t b, int64_t N)
{
    return a * N - a * (a + 1) / 2 + (b - a - 1);
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ======================= exported entry points ========================== */

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* cRMSD of one pair; R_out (row-major 3x3, may be NULL) receives the Kabsch
 * rotation that maps centred b onto centred a. */
int oracle_crmsd_pair(const float *A, const float *B, int64_t L, double *c_out, double *R_out)
{
    if (!A || !B || !c_out || L < 1) return ORACLE_EINVAL;
    double *ac = (double *)malloc(sizeof(double) * 3 * L);
    double *bc = (double *)malloc(sizeof(double) * 3 * L);
    if (!ac || !bc) { free(ac); free(bc); return ORACLE_EINVAL; }
    centre(A, L, ac);
    centre(B, L, bc);
    double R[3][3];
    int st = pair_from_centred(ac, bc, L, c_out, R);
    if (R_out && !st) memcpy(R_out, R, sizeof R);
    free(ac);
    free(bc);
    return st;
}

/* Condensed all-vs-all matrix: out[idx(a,b)] for a < b, idx = aN - a(a+1)/2 + b-a-1. */
int oracle_crmsd_allpairs(const float *X, int64_t N, int64_t L, double *out, int nthreads)
{
    if (!X || !out || N < 2 || L < 1) return ORACLE_EINVAL;
    double *xc = (double *)malloc(sizeof(double) * 3 * L * N);
    if (!xc) return ORACLE_EINVAL;
    for (int64_t a = 0; a < N; ++a) centre(X + 3 * L * a, L, xc + 3 * L * a);
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t a = 0; a < N - 1; ++a) {
        double R[3][3];
        for (int64_t b = a + 1; b < N; ++b) {
            double c = NAN;
            bad |= pair_from_centred(xc + 3 * L * a, xc + 3 * L * b, L, &c, R);
            out[condensed(a, b, N)] = c;
        }
    }
    free(xc);
    return bad ? ORACLE_ENOCONV : ORACLE_OK;
}

/* cRMSD for an explicit list of pairs (ia[k], ib[k]) in any order. */
int oracle_crmsd_pairs(const float *X, int64_t N, int64_t L, const int64_t *ia, const int64_t *ib,
                       int64_t npairs, double *out, int nthreads)
{
    if (!X || !ia || !ib || !out || N < 1 || L < 1 || npairs < 0) return ORACLE_EINVAL;
    for (int64_t k = 0; k < npairs; ++k)
        if (ia[k] < 0 || ia[k] >= N || ib[k] < 0 || ib[k] >= N) return ORACLE_EINVAL;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        double *ac = (double *)malloc(sizeof(double) * 3 * L);
        double *bc = (double *)malloc(sizeof(double) * 3 * L);
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < npairs; ++k) {
            double R[3][3], c = NAN;
            centre(X + 3 * L * ia[k], L, ac);
            centre(X + 3 * L * ib[k], L, bc);
            bad |= pair_from_centred(ac, bc, L, &c, R);
            out[k] = c;
        }
        free(ac);
        free(bc);
    }
    return bad ? ORACLE_ENOCONV : ORACLE_OK;
}

/* One-versus-reference: out[a] = cRMSD(model a, ref). */
int oracle_crmsd_vs_ref(const float *X, int64_t N, int64_t L, const float *ref, double *out, int nthreads)
{
    if (!X || !ref || !out || N < 1 || L < 1) return ORACLE_EINVAL;
    double *rc = (double *)malloc(sizeof(double) * 3 * L);
    if (!rc) return ORACLE_EINVAL;
    centre(ref, L, rc);
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        double *ac = (double *)malloc(sizeof(double) * 3 * L);
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < N; ++a) {
            double R[3][3], c = NAN;
            centre(X + 3 * L * a, L, ac);
            bad |= pair_from_centred(ac, rc, L, &c, R);
            out[a] = c;
        }
        free(ac);
    }
    free(rc);
    return bad ? ORACLE_ENOCONV : ORACLE_OK;
}

/* Gradient of sum_{a<b} w_ab cRMSD_ab with respect to every input coordinate.
 * w is condensed (length N(N-1)/2); grad is [N][L][3], overwritten.
 * Each model's gradient is assembled from its own side of every pair: for
 * model a and partner b, R is the rotation taking centred b onto centred a and
 * the term is w_ab (a_i - R b_i) / (L max(c_ab, eps)); then the centring's
 * chain rule subtracts the mean over atoms. */
int oracle_crmsd_grad(const float *X, int64_t N, int64_t L, const double *w, double eps,
                      double *grad, int nthreads)
{
    if (!X || !w || !grad || N < 2 || L < 1 || !(eps >= 0.0)) return ORACLE_EINVAL;
    double *xc = (double *)malloc(sizeof(double) * 3 * L * N);
    if (!xc) return ORACLE_EINVAL;
    for (int64_t a = 0; a < N; ++a) centre(X + 3 * L * a, L, xc + 3 * L * a);
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t a = 0; a < N; ++a) {
        double *g = grad + 3 * L * a;
        const double *ac = xc + 3 * L * a;
        for (int64_t j = 0; j < 3 * L; ++j) g[j] = 0.0;
        for (int64_t b = 0; b < N; ++b) {
            if (b == a) continue;
            const double *bc = xc + 3 * L * b;
            double R[3][3], c = NAN;
            bad |= pair_from_centred(ac, bc, L, &c, R);
            double wab = (a < b) ? w[condensed(a, b, N)] : w[condensed(b, a, N)];
            double coef = wab / ((double)L * fmax(c, eps));
            for (int64_t i = 0; i < L; ++i)
                for (int r = 0; r < 3; ++r) {
                    double rb = R[r][0] * bc[3 * i + 0] + R[r][1] * bc[3 * i + 1] + R[r][2] * bc[3 * i + 2];
                    g[3 * i + r] += coef * (ac[3 * i + r] - rb);
                }
        }
        /* chain rule through the centring: x_c = x - mean(x) */
        double m[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < L; ++i)
            for (int r = 0; r < 3; ++r) m[r] += g[3 * i + r];
        for (int64_t i = 0; i < L; ++i)
            for (int r = 0; r < 3; ++r) g[3 * i + r] -= m[r] / (double)L;
    }
    free(xc);
    return bad ? ORACLE_ENOCONV : ORACLE_OK;
}

/* Gradient rows: the same as oracle_crmsd_grad but only for the listed models
 * (rows[k], k < nrows), written to grad[k][L][3]; for spot checks at sizes where the full
 * gradient would take O(N^2 L) time. */
int oracle_crmsd_grad_rows(const float *X, int64_t N, int64_t L, const double *w, double eps,
                           const int64_t *rows, int64_t nrows, double *grad, int nthreads)
{
    if (!X || !w || !rows || !grad || N < 2 || L < 1 || nrows < 0 || !(eps >= 0.0)) return ORACLE_EINVAL;
    for (int64_t k = 0; k < nrows; ++k)
        if (rows[k] < 0 || rows[k] >= N) return ORACLE_EINVAL;
    int bad = 0;
    set_threads(nthreads);
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t a = rows[k];
        double *g = grad + 3 * L * k;
        double *ac = (double *)malloc(sizeof(double) * 3 * L);
        centre(X + 3 * L * a, L, ac);
        for (int64_t j = 0; j < 3 * L; ++j) g[j] = 0.0;
#pragma omp parallel reduction(| : bad)
        {
            double *bc = (double *)malloc(sizeof(double) * 3 * L);
            double *gl = (double *)calloc((size_t)(3 * L), sizeof(double));
#pragma omp for schedule(dynamic, 16)
            for (int64_t b = 0; b < N; ++b) {
                if (b == a) continue;
                double R[3][3], c = NAN;
                centre(X + 3 * L * b, L, bc);
                bad |= pair_from_centred(ac, bc, L, &c, R);
                double wab = (a < b) ? w[condensed(a, b, N)] : w[condensed(b, a, N)];
                double coef = wab / ((double)L * fmax(c, eps));
                for (int64_t i = 0; i < L; ++i)
                    for (int r = 0; r < 3; ++r) {
                        double rb = R[r][0] * bc[3 * i + 0] + R[r][1] * bc[3 * i + 1] + R[r][2] * bc[3 * i + 2];
                        gl[3 * i + r] += coef * (ac[3 * i + r] - rb);
                    }
            }
#pragma omp critical
            for (int64_t j = 0; j < 3 * L; ++j) g[j] += gl[j];
            free(bc);
            free(gl);
        }
        double m[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < L; ++i)
            for (int r = 0; r < 3; ++r) m[r] += g[3 * i + r];
        for (int64_t i = 0; i < L; ++i)
            for (int r = 0; r < 3; ++r) g[3 * i + r] -= m[r] / (double)L;
        free(ac);
    }
    return bad ? ORACLE_ENOCONV : ORACLE_OK;
}

/* The paper's closed form (eq. 2), FP64: eigenvalues of M^T M as roots of the
 * characteristic cubic, trigonometric (Viete) solution, S = sign(det M)
 * (S = +1 when det M = 0), negative eigenvalues and negative D clamped to 0. */
int oracle_crmsd_eq2(const float *A, const float *B, int64_t L, double *c_out)
{
    if (!A || !B || !c_out || L < 1) return ORACLE_EINVAL;
    double *ac = (double *)malloc(sizeof(double) * 3 * L);
    double *bc = (double *)malloc(sizeof(double) * 3 * L);
    if (!ac || !bc) { free(ac); free(bc); return ORACLE_EINVAL; }
    centre(A, L, ac);
    centre(B, L, bc);
    double M[3][3];
    covariance(ac, bc, L, M);
    double ra2 = 0.0, rb2 = 0.0;
    for (int64_t j = 0; j < 3 * L; ++j) { ra2 += ac[j] * ac[j]; rb2 += bc[j] * bc[j]; }
    ra2 /= (double)L;
    rb2 /= (double)L;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] /= (double)L;
    double S = det3(M) < 0.0 ? -1.0 : 1.0;
    double K[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            K[r][c] = M[0][r] * M[0][c] + M[1][r] * M[1][c] + M[2][r] * M[2][c];
    double c2 = K[0][0] + K[1][1] + K[2][2];
    double c1 = (K[0][0] * K[1][1] - K[0][1] * K[1][0]) + (K[0][0] * K[2][2] - K[0][2] * K[2][0])
              + (K[1][1] * K[2][2] - K[1][2] * K[2][1]);
    double c0 = det3(K);
    double m = c2 / 3.0;
    double p = c1 - 3.0 * m * m;
    double q = -2.0 * m * m * m + c1 * m - c0;
    double lam[3];
    if (p >= 0.0) {
        lam[0] = lam[1] = lam[2] = m;
    } else {
        double r = sqrt(-p / 3.0);
        double arg = (3.0 * q / (2.0 * p)) * sqrt(-3.0 / p);
        if (arg > 1.0) arg = 1.0;
        if (arg < -1.0) arg = -1.0;
        double th = acos(arg) / 3.0;
        for (int k = 0; k < 3; ++k) lam[k] = m + 2.0 * r * cos(th - 2.0 * M_PI * k / 3.0);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (lam[b] > lam[a]) { double t = lam[a]; lam[a] = lam[b]; lam[b] = t; }
    for (int k = 0; k < 3; ++k) if (lam[k] < 0.0) lam[k] = 0.0;
    double sig = sqrt(lam[0]) + sqrt(lam[1]) + S * sqrt(lam[2]);
    double D = ra2 + rb2 - 2.0 * sig;
    *c_out = sqrt(D > 0.0 ? D : 0.0);
    free(ac);
    free(bc);
    return ORACLE_OK;
}

/* ======================= GDT_TS, TM-score, MaxSub ======================= */
/*
 * Scores of a model against a reference after a search over superpositions (section
 * "Algorithms": GDT_TS eq. 3, TM-score eq. 4, MaxSub = TM-score with d0 = 3.5 A), by the
 * search the paper describes, in this order:
 *   1. seeds: every contiguous fragment of 4, L/4, L/2 and L atoms (lengths below 3 or above L
 *      dropped, repeated lengths taken once);
 *   2. for each seed, the whole model is superimposed on the reference by the optimal proper
 *      rotation and translation of the seed's atoms (Kabsch on their centred coordinates);
 *   3. that superposition is scored: d_i = |R b_i + t - a_i| for every atom, C_x = #{d_i < x}
 *      for x = 1, 2, 4, 8 A, the TM sum (1/L) sum_i 1 / (1 + (d_i/d0)^2) with
 *      d0 = max(1.24 (L - 15)^(1/3) - 1.8, 0.5) A and the same sum with d0 = 3.5 A (MaxSub);
 *   4. the atoms with d_i < 3.5 A are selected and the model is superimposed again on them,
 *      scored again, and so on, "until the number of selected atoms does not change in four
 *      iterations": the refinements stop once four refinements in a row have selected as many
 *      atoms as the superposition before them, when fewer than 3 atoms are selected, or after
 *      a bound of 20 refinements (the text gives none) where the count keeps changing. Where a
 *      refinement selects exactly the atoms it was fitted on, every later superposition is the
 *      same one, so the search stops there too (it cannot change any maximum);
 * and each score is the maximum over every superposition scored:
 *   GDT_TS = (max C_1 + max C_2 + max C_4 + max C_8) / (4 L), TM = max TM sum, MaxSub = max.
 */
static double tm_d0(int64_t L)
{
    const double d0 = 1.24 * cbrt((double)L - 15.0) - 1.8;
    return d0 > 0.5 ? d0 : 0.5;
}

/* R, t with R b_i + t ~ a_i from the atoms idx[0 .. n) (steps 2 and 4) */
static int fit_subset(const double *a, const double *b, const int64_t *idx, int64_t n, double *ac, double *bc,
                      double R[3][3], double t[3])
{
    double ma[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
    for (int64_t q = 0; q < n; ++q)
        for (int k = 0; k < 3; ++k) {
            ma[k] += a[3 * idx[q] + k];
            mb[k] += b[3 * idx[q] + k];
        }
    for (int k = 0; k < 3; ++k) {
        ma[k] /= (double)n;
        mb[k] /= (double)n;
    }
    for (int64_t q = 0; q < n; ++q)
        for (int k = 0; k < 3; ++k) {
            ac[3 * q + k] = a[3 * idx[q] + k] - ma[k];
            bc[3 * q + k] = b[3 * idx[q] + k] - mb[k];
        }
    int st = kabsch(ac, bc, n, R);
    if (st) return st;
    for (int r = 0; r < 3; ++r) t[r] = ma[r] - (R[r][0] * mb[0] + R[r][1] * mb[1] + R[r][2] * mb[2]);
    return ORACLE_OK;
}

#define GDT_STABLE 4       /* iterations without a change of the selected count that end a search */
#define GDT_MAX_REFINE 20  /* refinements at most */

/* out[0..3) = GDT_TS, TM-score, MaxSub of model b against reference a (L atoms each); the search
 * stops after `stable` refinements in a row without a change of the count, or `max_refine`. */
static int gdt_tm_one(const double *a, const double *b, int64_t L, int64_t *idx, int64_t *sel, double *ac,
                      double *bc, int stable, int max_refine, double out[3])
{
    const double cuts[4] = {1.0, 2.0, 4.0, 8.0};
    const double d0 = tm_d0(L), d0m = 3.5;
    int64_t best_c[4] = {0, 0, 0, 0};
    double best_tm = 0.0, best_ms = 0.0;
    int64_t lens[4] = {4, L / 4, L / 2, L};
    for (int li = 0; li < 4; ++li) {
        const int64_t len = lens[li];
        if (len < 3 || len > L) continue;
        int dup = 0;
        for (int lj = 0; lj < li; ++lj)
            if (lens[lj] == len) dup = 1;
        if (dup) continue;
        for (int64_t s0 = 0; s0 + len <= L; ++s0) {
            int64_t n = len, prev = -1;
            int same = 0;
            for (int64_t q = 0; q < n; ++q) idx[q] = s0 + q;
            for (int it = 0; it <= max_refine; ++it) {
                double R[3][3], t[3];
                int st = fit_subset(a, b, idx, n, ac, bc, R, t);
                if (st) return st;
                int64_t c[4] = {0, 0, 0, 0}, ns = 0;
                double tm = 0.0, ms = 0.0;
                for (int64_t i = 0; i < L; ++i) {
                    double d2 = 0.0;
                    for (int r = 0; r < 3; ++r) {
                        const double x = R[r][0] * b[3 * i] + R[r][1] * b[3 * i + 1] + R[r][2] * b[3 * i + 2] + t[r];
                        const double e = x - a[3 * i + r];
                        d2 += e * e;
                    }
                    const double d = sqrt(d2);
                    for (int k = 0; k < 4; ++k) c[k] += d < cuts[k];
                    tm += 1.0 / (1.0 + (d / d0) * (d / d0));
                    ms += 1.0 / (1.0 + (d / d0m) * (d / d0m));
                    if (d < 3.5) sel[ns++] = i;
                }
                for (int k = 0; k < 4; ++k)
                    if (c[k] > best_c[k]) best_c[k] = c[k];
                if (tm / (double)L > best_tm) best_tm = tm / (double)L;
                if (ms / (double)L > best_ms) best_ms = ms / (double)L;
                if (it == max_refine || ns < 3) break;
                same = (ns == prev) ? same + 1 : 0;
                if (same >= stable) break;
                if (ns == n) {  /* the atoms it was fitted on: the same superposition from here on */
                    int64_t q = 0;
                    while (q < n && idx[q] == sel[q]) ++q;
                    if (q == n) break;
                }
                prev = ns;
                n = ns;
                for (int64_t q = 0; q < n; ++q) idx[q] = sel[q];
            }
        }
    }
    out[0] = (double)(best_c[0] + best_c[1] + best_c[2] + best_c[3]) / (4.0 * (double)L);
    out[1] = best_tm;
    out[2] = best_ms;
    return ORACLE_OK;
}

/* GDT_TS, TM-score and MaxSub of every model against the reference, out[3 a + {0,1,2}], with the
 * search's stop rule as parameters: stable = 4, max_refine = 20 is the reading above; stable = 1,
 * max_refine = 4 stops at the first repeated count or after four refinements (a shorter reading of
 * the same sentence, kept for the tests that tell the two apart). */
int oracle_gdt_tm_vs_ref_rule(const float *X, int64_t N, int64_t L, const float *ref, double *out, int nthreads,
                              int stable, int max_refine)
{
    if (!X || !ref || !out || N < 1 || L < 3 || stable < 1 || max_refine < 0) return ORACLE_EINVAL;
    double *a = (double *)malloc(sizeof(double) * 3 * L);
    if (!a) return ORACLE_EINVAL;
    for (int64_t t = 0; t < 3 * L; ++t) a[t] = (double)ref[t];
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        double *b = (double *)malloc(sizeof(double) * 3 * L);
        double *ac = (double *)malloc(sizeof(double) * 3 * L);
        double *bc = (double *)malloc(sizeof(double) * 3 * L);
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * L);
        int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * L);
        if (!b || !ac || !bc || !idx || !sel) bad = 1;
#pragma omp for schedule(dynamic, 1)
        for (int64_t m = 0; m < N; ++m) {
            if (bad) continue;
            for (int64_t t = 0; t < 3 * L; ++t) b[t] = (double)X[3 * L * m + t];
            bad |= gdt_tm_one(a, b, L, idx, sel, ac, bc, stable, max_refine, out + 3 * m);
        }
        free(b);
        free(ac);
        free(bc);
        free(idx);
        free(sel);
    }
    free(a);
    return bad ? ORACLE_ENOCONV : ORACLE_OK;
}

/* GDT_TS, TM-score and MaxSub with the stop rule of the search described above. */
int oracle_gdt_tm_vs_ref(const float *X, int64_t N, int64_t L, const float *ref, double *out, int nthreads)
{
    return oracle_gdt_tm_vs_ref_rule(X, N, L, ref, out, nthreads, GDT_STABLE, GDT_MAX_REFINE);
}

/*
 * drmsd_oracle.c -- FP64 CPU oracle for all-versus-all dRMSD.
 *
 * TEST INFRASTRUCTURE, like crmsd_oracle.c: the plain, slow reference that the
 * CUDA path is checked against; only the tests, the smoke check and the bench's
 * CPU-baseline leg may load it. It shares no code, header, helper or constant
 * with the CUDA path.
 *
 * What it computes (ClusCo, section "Algorithms", eq. 5, the distance RMSD):
 *
 *   dRMSD(A, B) = sqrt( 2 / (L (L - 1)) * sum_{i < j} (d^A_ij - d^B_ij)^2 )
 *
 * with d^A_ij = |a_i - a_j| the Euclidean distance between atoms i and j of
 * model A, over L >= 2 matched atoms. Steps, in this order, all in FP64 (the
 * FP32 coordinates are promoted exactly):
 *   1. for each model, the L (L - 1) / 2 intra-model distances d_ij, i < j;
 *   2. the sum over i < j of the squared differences of the two models'
 *      distances, formed directly (no expansion into squares and a cross
 *      term, so nothing cancels as dRMSD -> 0);
 *   3. times 2 / (L (L - 1)), square root.
 * Non-finite coordinates give NaN. No superposition is involved, so the score
 * is blind to a mirror image (the paper's remark on chirality).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

/* step 1: the distances of one model, d[k] for i < j in row-major order
 * k = i (2L - i - 1) / 2 + (j - i - 1) */
static void distances(const float *x, int64_t L, double *d)
{
    int64_t k = 0;
    for (int64_t i = 0; i < L; ++i)
        for (int64_t j = i + 1; j < L; ++j) {
            double s = 0.0;
            for (int ax = 0; ax < 3; ++ax) {
                const double t = (double)x[3 * i + ax] - (double)x[3 * j + ax];
                s += t * t;
            }
            d[k++] = sqrt(s);
        }
}

/* steps 2 and 3 */
static double drmsd_from_distances(const double *da, const double *db, int64_t L)
{
    const int64_t K = L * (L - 1) / 2;
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        const double t = da[k] - db[k];
        s += t * t;
    }
    return sqrt(2.0 * s / ((double)L * (double)(L - 1)));
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

/* dRMSD of one pair of models of L atoms. */
int oracle_drmsd_pair(const float *A, const float *B, int64_t L, double *out)
{
    if (!A || !B || !out || L < 2) return ORACLE_EINVAL;
    const int64_t K = L * (L - 1) / 2;
    double *da = (double *)malloc(sizeof(double) * K);
    double *db = (double *)malloc(sizeof(double) * K);
    if (!da || !db) { free(da); free(db); return ORACLE_EINVAL; }
    distances(A, L, da);
    distances(B, L, db);
    *out = drmsd_from_distances(da, db, L);
    free(da);
    free(db);
    return ORACLE_OK;
}

/* Condensed all-vs-all matrix: out[idx(a,b)] for a < b, idx = aN - a(a+1)/2 + b-a-1.
 * Holds every model's distances (8 N L (L - 1) / 2 bytes). */
int oracle_drmsd_allpairs(const float *X, int64_t N, int64_t L, double *out, int nthreads)
{
    if (!X || !out || N < 2 || L < 2) return ORACLE_EINVAL;
    const int64_t K = L * (L - 1) / 2;
    double *d = (double *)malloc(sizeof(double) * K * N);
    if (!d) return ORACLE_EINVAL;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < N; ++a) distances(X + 3 * L * a, L, d + K * a);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < N - 1; ++a)
        for (int64_t b = a + 1; b < N; ++b) out[condensed(a, b, N)] = drmsd_from_distances(d + K * a, d + K * b, L);
    free(d);
    return ORACLE_OK;
}

/* dRMSD for an explicit list of pairs (ia[k], ib[k]) in any order; distances are
 * recomputed per pair, so memory stays O(L^2) per thread. */
int oracle_drmsd_pairs(const float *X, int64_t N, int64_t L, const int64_t *ia, const int64_t *ib,
                       int64_t npairs, double *out, int nthreads)
{
    if (!X || !ia || !ib || !out || N < 1 || L < 2 || npairs < 0) return ORACLE_EINVAL;
    for (int64_t k = 0; k < npairs; ++k)
        if (ia[k] < 0 || ia[k] >= N || ib[k] < 0 || ib[k] >= N) return ORACLE_EINVAL;
    const int64_t K = L * (L - 1) / 2;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        double *da = (double *)malloc(sizeof(double) * K);
        double *db = (double *)malloc(sizeof(double) * K);
        if (!da || !db) bad = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < npairs; ++k) {
            if (!da || !db) continue;
            distances(X + 3 * L * ia[k], L, da);
            distances(X + 3 * L * ib[k], L, db);
            out[k] = drmsd_from_distances(da, db, L);
        }
        free(da);
        free(db);
    }
    return bad ? ORACLE_EINVAL : ORACLE_OK;
}

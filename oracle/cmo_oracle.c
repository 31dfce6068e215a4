/*
 * cmo_oracle.c -- CPU oracle for all-versus-all contact map overlap (CMO).
 *
 * TEST INFRASTRUCTURE, like crmsd_oracle.c: only the tests, the smoke check and
 * the bench's CPU-baseline leg may load it; it shares no code, header, helper or
 * constant with the CUDA path.
 *
 * What it computes (ClusCo, section "Algorithms", eq. 6 and eq. 7):
 *   contact map  C_ij = 1 if |x_i - x_j| < cutoff, else 0, over the atom pairs i < j;
 *   score        S(A, B) = 100 * 2 n(A and B) / (n(A) + n(B)),
 * with n(.) the number of contacts (of a map, or of both maps at once).
 * Steps, in this order:
 *   1. each model's contact map, the test |x_i - x_j| < cutoff taken in FP64 from the given
 *      FP32 coordinates: the differences and their squares are exact in FP64, so the squared
 *      distance carries one rounding of its sum (2^-53 relative) and the strict comparison
 *      with cutoff^2 (exact) decides the definition's inequality except for distances within
 *      that rounding of the cutoff (compiled with contraction off, as written);
 *   2. the counts n(A), n(B) and n(A and B), exact integers;
 *   3. the score in FP64. Where n(A) + n(B) = 0 (neither model has a contact) the
 *      score is taken as 0.
 * A model with a non-finite coordinate scores NaN against every model.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

static int finite_model(const float *x, int64_t L)
{
    for (int64_t t = 0; t < 3 * L; ++t)
        if (!isfinite(x[t])) return 0;
    return 1;
}

/* step 1: the contact map of one model, c[k] for i < j in row-major order */
static void contact_map(const float *x, int64_t L, float cutoff, unsigned char *c)
{
    const double cut2 = (double)cutoff * (double)cutoff;
    int64_t k = 0;
    for (int64_t i = 0; i < L; ++i)
        for (int64_t j = i + 1; j < L; ++j) {
            const double dx = (double)x[3 * i] - (double)x[3 * j];
            const double dy = (double)x[3 * i + 1] - (double)x[3 * j + 1];
            const double dz = (double)x[3 * i + 2] - (double)x[3 * j + 2];
            const double d2 = dx * dx + dy * dy + dz * dz;
            c[k++] = d2 < cut2 ? 1 : 0;
        }
}

/* steps 2 and 3 */
static double score(const unsigned char *ca, const unsigned char *cb, int64_t K)
{
    int64_t na = 0, nb = 0, nab = 0;
    for (int64_t k = 0; k < K; ++k) {
        na += ca[k];
        nb += cb[k];
        nab += ca[k] & cb[k];
    }
    if (na + nb == 0) return 0.0;
    return 100.0 * 2.0 * (double)nab / (double)(na + nb);
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

/* Contact counts of one model (n(A)) and of one pair (n(A and B)), for pins. */
int oracle_cmo_counts(const float *A, const float *B, int64_t L, float cutoff, int64_t *na, int64_t *nb,
                      int64_t *nab)
{
    if (!A || !B || !na || !nb || !nab || L < 2) return ORACLE_EINVAL;
    const int64_t K = L * (L - 1) / 2;
    unsigned char *ca = (unsigned char *)malloc(K), *cb = (unsigned char *)malloc(K);
    if (!ca || !cb) { free(ca); free(cb); return ORACLE_EINVAL; }
    contact_map(A, L, cutoff, ca);
    contact_map(B, L, cutoff, cb);
    *na = *nb = *nab = 0;
    for (int64_t k = 0; k < K; ++k) {
        *na += ca[k];
        *nb += cb[k];
        *nab += ca[k] & cb[k];
    }
    free(ca);
    free(cb);
    return ORACLE_OK;
}

/* CMO score of one pair of models. */
int oracle_cmo_pair(const float *A, const float *B, int64_t L, float cutoff, double *out)
{
    if (!A || !B || !out || L < 2) return ORACLE_EINVAL;
    if (!finite_model(A, L) || !finite_model(B, L)) {
        *out = NAN;
        return ORACLE_OK;
    }
    const int64_t K = L * (L - 1) / 2;
    unsigned char *ca = (unsigned char *)malloc(K), *cb = (unsigned char *)malloc(K);
    if (!ca || !cb) { free(ca); free(cb); return ORACLE_EINVAL; }
    contact_map(A, L, cutoff, ca);
    contact_map(B, L, cutoff, cb);
    *out = score(ca, cb, K);
    free(ca);
    free(cb);
    return ORACLE_OK;
}

/* Condensed all-vs-all matrix: out[idx(a,b)] for a < b. Holds every model's map (N K bytes). */
int oracle_cmo_allpairs(const float *X, int64_t N, int64_t L, float cutoff, double *out, int nthreads)
{
    if (!X || !out || N < 2 || L < 2) return ORACLE_EINVAL;
    const int64_t K = L * (L - 1) / 2;
    unsigned char *c = (unsigned char *)malloc((size_t)(K * N));
    int *fin = (int *)malloc(sizeof(int) * N);
    if (!c || !fin) { free(c); free(fin); return ORACLE_EINVAL; }
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < N; ++a) {
        fin[a] = finite_model(X + 3 * L * a, L);
        contact_map(X + 3 * L * a, L, cutoff, c + K * a);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < N - 1; ++a)
        for (int64_t b = a + 1; b < N; ++b)
            out[condensed(a, b, N)] = (fin[a] && fin[b]) ? score(c + K * a, c + K * b, K) : NAN;
    free(c);
    free(fin);
    return ORACLE_OK;
}

/* CMO for an explicit list of pairs (ia[k], ib[k]) in any order. */
int oracle_cmo_pairs(const float *X, int64_t N, int64_t L, float cutoff, const int64_t *ia, const int64_t *ib,
                     int64_t npairs, double *out, int nthreads)
{
    if (!X || !ia || !ib || !out || N < 1 || L < 2 || npairs < 0) return ORACLE_EINVAL;
    for (int64_t k = 0; k < npairs; ++k)
        if (ia[k] < 0 || ia[k] >= N || ib[k] < 0 || ib[k] >= N) return ORACLE_EINVAL;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t k = 0; k < npairs; ++k)
        bad |= oracle_cmo_pair(X + 3 * L * ia[k], X + 3 * L * ib[k], L, cutoff, out + k);
    return bad ? ORACLE_EINVAL : ORACLE_OK;
}

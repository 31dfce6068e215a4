// rotation.cuh -- optimal rotation from a covariance by Horn's quaternion form, FP32 or FP64.
//
// With H = sum_i a_i b_i^T (centred), every unit quaternion q gives a rotation R(q) with
//   sum_i a_i . R(q) b_i = sum_jk R(q)_jk H_jk = q^T K q,
// K the symmetric traceless 4x4 key matrix below. The largest eigenvalue of K is
// Sigma = s1 + s2 + S s3 (the same quantity as in eq. 2) and its eigenvector gives the
// rotation that superposes b onto a. Two routes: the adjugate of K - Sigma I (a few hundred
// operations; its columns are proportional to the eigenvector) and, where that eigenvalue is
// repeated and the adjugate vanishes, cyclic Jacobi sweeps (well defined there). The hot
// paths take the rotation from the closed form dSigma/dM in epilogue.cuh and come here only
// near a double root.
#pragma once

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T sel4(int i, T a, T b, T c, T d)
{
    return i == 0 ? a : (i == 1 ? b : (i == 2 ? c : d));
}

// Rotation matrix (row-major) of the quaternion q scaled by inv (inv = 1/|q|).
template <typename T>
__device__ __forceinline__ void quat_to_rotation(const T q[4], T inv, T R[9])
{
    const T w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    R[0] = w * w + x * x - y * y - z * z;
    R[1] = T(2) * (x * y - w * z);
    R[2] = T(2) * (x * z + w * y);
    R[3] = T(2) * (x * y + w * z);
    R[4] = w * w - x * x + y * y - z * z;
    R[5] = T(2) * (y * z - w * x);
    R[6] = T(2) * (x * z - w * y);
    R[7] = T(2) * (y * z + w * x);
    R[8] = w * w - x * x - y * y + z * z;
}

// Adjugate of a 4x4 matrix by Laplace expansion along rows (0,1) against rows (2,3):
// twelve 2x2 minors, then each cofactor as three products. adj[i][j] = (-1)^(i+j) M_ji.
template <typename T>
__device__ __forceinline__ void adjugate4(const T A[4][4], T adj[4][4])
{
    const T s0 = A[0][0] * A[1][1] - A[1][0] * A[0][1];
    const T s1 = A[0][0] * A[1][2] - A[1][0] * A[0][2];
    const T s2 = A[0][0] * A[1][3] - A[1][0] * A[0][3];
    const T s3 = A[0][1] * A[1][2] - A[1][1] * A[0][2];
    const T s4 = A[0][1] * A[1][3] - A[1][1] * A[0][3];
    const T s5 = A[0][2] * A[1][3] - A[1][2] * A[0][3];
    const T c5 = A[2][2] * A[3][3] - A[3][2] * A[2][3];
    const T c4 = A[2][1] * A[3][3] - A[3][1] * A[2][3];
    const T c3 = A[2][1] * A[3][2] - A[3][1] * A[2][2];
    const T c2 = A[2][0] * A[3][3] - A[3][0] * A[2][3];
    const T c1 = A[2][0] * A[3][2] - A[3][0] * A[2][2];
    const T c0 = A[2][0] * A[3][1] - A[3][0] * A[2][1];
    adj[0][0] = A[1][1] * c5 - A[1][2] * c4 + A[1][3] * c3;
    adj[0][1] = -A[0][1] * c5 + A[0][2] * c4 - A[0][3] * c3;
    adj[0][2] = A[3][1] * s5 - A[3][2] * s4 + A[3][3] * s3;
    adj[0][3] = -A[2][1] * s5 + A[2][2] * s4 - A[2][3] * s3;
    adj[1][0] = -A[1][0] * c5 + A[1][2] * c2 - A[1][3] * c1;
    adj[1][1] = A[0][0] * c5 - A[0][2] * c2 + A[0][3] * c1;
    adj[1][2] = -A[3][0] * s5 + A[3][2] * s2 - A[3][3] * s1;
    adj[1][3] = A[2][0] * s5 - A[2][2] * s2 + A[2][3] * s1;
    adj[2][0] = A[1][0] * c4 - A[1][1] * c2 + A[1][3] * c0;
    adj[2][1] = -A[0][0] * c4 + A[0][1] * c2 - A[0][3] * c0;
    adj[2][2] = A[3][0] * s4 - A[3][1] * s2 + A[3][3] * s0;
    adj[2][3] = -A[2][0] * s4 + A[2][1] * s2 - A[2][3] * s0;
    adj[3][0] = -A[1][0] * c3 + A[1][1] * c1 - A[1][2] * c0;
    adj[3][1] = A[0][0] * c3 - A[0][1] * c1 + A[0][2] * c0;
    adj[3][2] = -A[3][0] * s3 + A[3][1] * s1 - A[3][2] * s0;
    adj[3][3] = A[2][0] * s3 - A[2][1] * s1 + A[2][2] * s0;
}

// R (row-major) maximising sum_i a_i . R b_i, given H (row-major) and lam = largest
// eigenvalue of K(H) (any consistent scaling of H and lam): every column of adj(K - lam I) is
// proportional to the top eigenvector q, with a norm near the product of the three eigenvalue
// gaps (P'(Sigma) for the quartic of eq. 2's Sigma). Returns false, leaving R unset, when that
// product is below tol * lam^3 (a (near-)repeated top eigenvalue: rank <= 1 covariance, or
// S = -1 with s2 = s3), where the adjugate carries no direction; rotation_jacobi4 then.
template <typename T>
__device__ __forceinline__ bool horn_rotation(const T H[9], T lam, T tol, T R[9])
{
    T A[4][4];
    A[0][0] = H[0] + H[4] + H[8] - lam;
    A[1][1] = H[0] - H[4] - H[8] - lam;
    A[2][2] = -H[0] + H[4] - H[8] - lam;
    A[3][3] = -H[0] - H[4] + H[8] - lam;
    A[0][1] = A[1][0] = H[7] - H[5];
    A[0][2] = A[2][0] = H[2] - H[6];
    A[0][3] = A[3][0] = H[3] - H[1];
    A[1][2] = A[2][1] = H[1] + H[3];
    A[1][3] = A[3][1] = H[2] + H[6];
    A[2][3] = A[3][2] = H[5] + H[7];
    // the column with the largest diagonal entry (all diagonal entries share one sign),
    // selected without indexing
    T adj[4][4];
    adjugate4(A, adj);
    int jb = 0;
    T best = fabs(adj[0][0]);
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        const T v = fabs(adj[j][j]);
        if (v > best) {
            best = v;
            jb = j;
        }
    }
    const T l3 = fabs(lam) * lam * lam;
    if (!(best > tol * l3) || !isfinite(best)) return false;
    T q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = sel4(jb, adj[k][0], adj[k][1], adj[k][2], adj[k][3]);
    const T n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    quat_to_rotation(q, rsqrt_t(n2), R);
    return true;
}

// One Jacobi rotation of the symmetric 4x4 matrix A in the (p, q) plane, annihilating A[p][q]
// (the symmetric Schur decomposition step), with the eigenvector matrix V updated alongside.
template <typename T, int p, int q>
__device__ __forceinline__ void jacobi_rotate(T (&A)[4][4], T (&V)[4][4])
{
    const T apq = A[p][q];
    if (!(fabs(apq) > T(1e-30) * (fabs(A[p][p]) + fabs(A[q][q])) + T(1e-37))) return;
    const T theta = (A[q][q] - A[p][p]) / (T(2) * apq);
    const T th2 = theta * theta;
    T t;
    if (isinf(th2))
        t = T(0.5) / theta;  // |theta| huge: t ~ 1/(2 theta)
    else
        t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(th2 + T(1)));
    const T c = rsqrt_t(t * t + T(1)), s = t * c;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k == p || k == q) continue;
        const T akp = A[k][p], akq = A[k][q];
        A[k][p] = A[p][k] = c * akp - s * akq;
        A[k][q] = A[q][k] = s * akp + c * akq;
    }
    A[p][p] -= t * apq;
    A[q][q] += t * apq;
    A[p][q] = A[q][p] = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
    }
}

// The same rotation from a full eigen-decomposition of K(H) by cyclic Jacobi sweeps: robust
// where the largest eigenvalue of K is (nearly) repeated -- a covariance of rank <= 1, or
// S = -1 with s2 = s3 -- where the adjugate above vanishes. There the optimal rotation is not
// unique and any unit vector of the top eigenspace gives one of them (the same superposed
// residuals for a rank-1 covariance). Used for the rare blocks the closed forms flag.
template <typename T, int SWEEPS>
__device__ __forceinline__ void rotation_jacobi4(const T H[9], T R[9])
{
    T A[4][4], V[4][4];
    A[0][0] = H[0] + H[4] + H[8];
    A[1][1] = H[0] - H[4] - H[8];
    A[2][2] = -H[0] + H[4] - H[8];
    A[3][3] = -H[0] - H[4] + H[8];
    A[0][1] = A[1][0] = H[7] - H[5];
    A[0][2] = A[2][0] = H[2] - H[6];
    A[0][3] = A[3][0] = H[3] - H[1];
    A[1][2] = A[2][1] = H[1] + H[3];
    A[1][3] = A[3][1] = H[2] + H[6];
    A[2][3] = A[3][2] = H[5] + H[7];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) V[i][j] = (i == j) ? T(1) : T(0);
#pragma unroll 1
    for (int sw = 0; sw < SWEEPS; ++sw) {
        jacobi_rotate<T, 0, 1>(A, V);
        jacobi_rotate<T, 0, 2>(A, V);
        jacobi_rotate<T, 0, 3>(A, V);
        jacobi_rotate<T, 1, 2>(A, V);
        jacobi_rotate<T, 1, 3>(A, V);
        jacobi_rotate<T, 2, 3>(A, V);
    }
    int kb = 0;
    T best = A[0][0];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        if (A[k][k] > best) {
            best = A[k][k];
            kb = k;
        }
    }
    T q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = sel4(kb, V[k][0], V[k][1], V[k][2], V[k][3]);
    const T n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > T(0)) || !isfinite(n2)) {
        R[0] = R[4] = R[8] = T(1);
        R[1] = R[2] = R[3] = R[5] = R[6] = R[7] = T(0);
        return;
    }
    quat_to_rotation(q, rsqrt_t(n2), R);
}

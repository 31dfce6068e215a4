// rotation.cuh -- optimal rotation from a covariance (Horn's quaternion form), FP32 or FP64.
//
// With H = sum_i a_i b_i^T (centred), every unit quaternion q gives a rotation R(q) with
//   sum_i a_i . R(q) b_i = sum_jk R(q)_jk H_jk = q^T K q,
// K the symmetric traceless 4x4 matrix below. The largest eigenvalue of K is
// Sigma = s1 + s2 + S s3 (the same quantity as in eq. 2) and its eigenvector gives the
// rotation that superposes b onto a. The eigenvector is read off the adjugate of
// K - Sigma I (rank 3): every column of adj is proportional to q; the column with the
// largest diagonal entry is the best conditioned.
#pragma once

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T sel4(int i, T a, T b, T c, T d)
{
    return i == 0 ? a : (i == 1 ? b : (i == 2 ? c : d));
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
// eigenvalue of K(H) (any consistent scaling of H and lam). Returns false when the
// eigenvector is undetermined (K - lam I of rank < 3 to working precision).
template <typename T>
__device__ __forceinline__ bool horn_rotation(const T H[9], T lam, T R[9])
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
    // every column of adj(K - lam I) is proportional to q; take the one with the largest
    // diagonal entry (all diagonal entries share one sign), selected without indexing
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
    T q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = sel4(jb, adj[k][0], adj[k][1], adj[k][2], adj[k][3]);
    const T n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > T(0)) || !isfinite(n2)) {
        R[0] = R[4] = R[8] = T(1);
        R[1] = R[2] = R[3] = R[5] = R[6] = R[7] = T(0);
        return false;
    }
    const T inv = rsqrt_t(n2);
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
    return true;
}

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

template <typename T>
__device__ __forceinline__ T det3_rows(const T A[4][4], int r0, int r1, int r2, int c0, int c1, int c2)
{
    return A[r0][c0] * (A[r1][c1] * A[r2][c2] - A[r1][c2] * A[r2][c1])
         - A[r0][c1] * (A[r1][c0] * A[r2][c2] - A[r1][c2] * A[r2][c0])
         + A[r0][c2] * (A[r1][c0] * A[r2][c1] - A[r1][c1] * A[r2][c0]);
}

// Cofactor C_jk of the 4x4 matrix A.
template <typename T>
__device__ __forceinline__ T cofactor4(const T A[4][4], int j, int k)
{
    int r[3], c[3];
    int n = 0;
    for (int i = 0; i < 4; ++i)
        if (i != j) r[n++] = i;
    n = 0;
    for (int i = 0; i < 4; ++i)
        if (i != k) c[n++] = i;
    const T d = det3_rows(A, r[0], r[1], r[2], c[0], c[1], c[2]);
    return ((j + k) & 1) ? -d : d;
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
    // adj_jj = cofactor C_jj >= 0 up to rounding; pick the largest
    int jb = 0;
    T best = cofactor4(A, 0, 0);
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        const T v = cofactor4(A, j, j);
        if (fabs(v) > fabs(best)) {
            best = v;
            jb = j;
        }
    }
    T q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = (k == jb) ? best : cofactor4(A, jb, k);
    const T n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > T(0)) || !isfinite(n2)) {
        R[0] = R[4] = R[8] = T(1);
        R[1] = R[2] = R[3] = R[5] = R[6] = R[7] = T(0);
        return false;
    }
    const T inv = T(1) / sqrt(n2);
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

"""Test helpers: condensed indexing and error bounds (no cRMSD arithmetic)."""
import numpy as np


def condensed_index(a, b, N):
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    return a * N - a * (a + 1) // 2 + (b - a - 1)


def all_pairs(N):
    a, b = np.triu_indices(N, 1)
    return a.astype(np.int64), b.astype(np.int64)


def sample_pairs(N, n, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, N, size=4 * n)
    b = rng.integers(0, N, size=4 * n)
    keep = a != b
    a, b = a[keep][:n], b[keep][:n]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    return lo.astype(np.int64), hi.astype(np.int64)


def gyration_sums(X):
    """G_a = sum_i |x_i - mean|^2 in FP64 (used only to scale error bounds)."""
    x = X.astype(np.float64)
    x = x - x.mean(axis=1, keepdims=True)
    return (x * x).sum(axis=(1, 2))


def c_error_bound(c_ref, Ga, Gb, L, rel_c2, floor=0.0):
    """Bound on |c_gpu - c_ref| from an absolute error rel_c2 * (Ga+Gb)/L on c^2."""
    d2 = rel_c2 * (Ga + Gb) / L
    c = np.asarray(c_ref, dtype=np.float64)
    return np.minimum(d2 / np.maximum(c, 1e-300), np.sqrt(d2)) + floor


def contact_band(X, cutoff, rel=2.0 ** -20):
    """Per model, the number of atom pairs i < j whose FP64 squared distance lies within
    rel * cutoff^2 of cutoff^2: the pairs where a contact test evaluated in FP32 (about 5 ulp of
    rounding in the differences, their squares and the sum) may decide otherwise than FP64."""
    X = np.asarray(X, dtype=np.float64)
    L = X.shape[1]
    i, j = np.triu_indices(L, 1)
    c2 = float(np.float32(cutoff)) ** 2
    out = np.empty(X.shape[0], dtype=np.int64)
    for m in range(X.shape[0]):
        d2 = ((X[m, i] - X[m, j]) ** 2).sum(axis=1)
        out[m] = int((np.abs(d2 - c2) <= rel * c2).sum())
    return out


def cmo_bounds(na, nb, nab, ka, kb):
    """Interval of 200 n'(A and B) / (n'(A) + n'(B)) when up to ka contacts of A and kb of B may be
    decided the other way (each changes n(A) or n(B) by one and n(A and B) by at most one)."""
    k = ka + kb
    lo_den = max(na + nb - k, 1)
    lo = 200.0 * max(nab - k, 0) / (na + nb + k) if na + nb + k > 0 else 0.0
    hi = min(100.0, 200.0 * (nab + k) / lo_den)
    return lo, hi

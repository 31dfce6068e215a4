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

"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every expected value comes from a
closed form derived by hand (tests/golden/closed_forms.txt), from an
independent formulation (eq. 2 of the paper solved with numpy's symmetric
eigensolver, brute-force rotation search), from an invariance of the metric,
or from finite differences of the oracle's own value function.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1302_4000_b300 import ensembles as E

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def read_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, L, a, b, val, _why = [f.strip() for f in line.split("|", 5)]
        A = np.array([[float(v) for v in r.split()] for r in a.split(";")], dtype=np.float32)
        B = np.array([[float(v) for v in r.split()] for r in b.split(";")], dtype=np.float32)
        assert A.shape == B.shape == (int(L), 3)
        cases.append((name, A, B, float(val)))
    return cases


def eq2_numpy(A, B):
    """Eq. 2 with the eigenvalues of M^T M from numpy's symmetric eigensolver."""
    a = A.astype(np.float64) - A.astype(np.float64).mean(0)
    b = B.astype(np.float64) - B.astype(np.float64).mean(0)
    L = a.shape[0]
    M = a.T @ b / L
    lam = np.clip(np.sort(np.linalg.eigvalsh(M.T @ M))[::-1], 0.0, None)
    S = -1.0 if np.linalg.det(M) < 0 else 1.0
    D = (a * a).sum() / L + (b * b).sum() / L - 2.0 * (np.sqrt(lam[0]) + np.sqrt(lam[1]) + S * np.sqrt(lam[2]))
    return np.sqrt(max(D, 0.0))


def rms_after(R, A, B):
    a = A.astype(np.float64) - A.astype(np.float64).mean(0)
    b = B.astype(np.float64) - B.astype(np.float64).mean(0)
    return np.sqrt(((a - b @ R.T) ** 2).sum() / a.shape[0])


def quat_to_R(q):
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


@pytest.mark.parametrize("case", read_golden(), ids=lambda c: c[0])
def test_closed_forms(case):
    _, A, B, expect = case
    c, R = oracle.crmsd_pair(A, B)
    assert abs(c - expect) <= 1e-12 * max(1.0, expect)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12  # a proper rotation


def test_eq2_agrees_with_kabsch():
    """Eq. 2 (independent eigensolver) reaches the Kabsch optimum (exact reading of P eq. 2)."""
    rng = np.random.default_rng(1)
    e = E.config0()
    worst = 0.0
    for _ in range(300):
        i, j = rng.choice(e.N, 2, replace=False)
        c, _ = oracle.crmsd_pair(e.coords[i], e.coords[j])
        worst = max(worst, abs(c - eq2_numpy(e.coords[i], e.coords[j])))
        # the paper's cubic route (restated in the oracle library) agrees as well
        assert abs(oracle.crmsd_eq2_pair(e.coords[i], e.coords[j]) - c) < 1e-9
    assert worst < 1e-10


def test_rigid_motion_invariance():
    """c(A, QA + t) is bounded by the FP32 cast of QA + t (metric property)."""
    rng = np.random.default_rng(2)
    e = E.config0()
    for k in range(20):
        A = e.coords[k]
        Q = E.haar_rotations(1, rng)[0]
        t = rng.uniform(-50, 50, 3)
        Bx = A.astype(np.float64) @ Q.T + t
        B = Bx.astype(np.float32)
        cast = np.sqrt(((B.astype(np.float64) - Bx) ** 2).sum() / A.shape[0])
        c, _ = oracle.crmsd_pair(A, B)
        assert c <= cast + 1e-12
        # and c(A, Q B' + t) = c(A, B') up to the same kind of bound
        C = e.coords[(k + 1) % e.N]
        Cx = C.astype(np.float64) @ Q.T + t
        C2 = Cx.astype(np.float32)
        cast2 = np.sqrt(((C2.astype(np.float64) - Cx) ** 2).sum() / A.shape[0])
        assert abs(oracle.crmsd_pair(A, C2)[0] - oracle.crmsd_pair(A, C)[0]) <= cast2 + 1e-12


def test_mirror_image_closed_form():
    """B = A diag(1,1,-1): S = -1 and cRMSD = 2 sqrt(mu_min / L), mu = gyration-tensor eigenvalues."""
    e = E.config0()
    for k in range(10):
        A = e.coords[k]
        B = (A * np.array([1, 1, -1], dtype=np.float32)).astype(np.float32)
        a = A.astype(np.float64) - A.astype(np.float64).mean(0)
        mu = np.linalg.eigvalsh(a.T @ a)
        expect = 2.0 * np.sqrt(mu[0] / A.shape[0])
        c, _ = oracle.crmsd_pair(A, B)
        assert expect > 1.0
        assert abs(c - expect) < 1e-10 * expect


def test_symmetry_triangle_nonnegativity():
    e = E.config0()
    X = e.coords[:10]
    D = np.zeros((10, 10))
    for i in range(10):
        for j in range(10):
            D[i, j] = oracle.crmsd_pair(X[i], X[j])[0]
    assert np.all(D >= 0)
    assert np.max(np.abs(D - D.T)) < 1e-11
    assert np.max(np.abs(np.diag(D))) < 1e-12
    for i in range(10):
        for j in range(10):
            for k in range(10):
                assert D[i, k] <= D[i, j] + D[j, k] + 1e-10


def test_scaled_copy_and_translation():
    e = E.config0()
    A = e.coords[3]
    a = A.astype(np.float64) - A.astype(np.float64).mean(0)
    RA = np.sqrt((a * a).sum() / A.shape[0])
    for s in (0.5, 2.0, 4.0):  # powers of two: the FP32 scaling is exact
        c, _ = oracle.crmsd_pair(A, (A * np.float32(s)).astype(np.float32))
        assert abs(c - abs(1 - s) * RA) < 1e-9 * RA
    c, _ = oracle.crmsd_pair(A, (A + np.float32(16.0)).astype(np.float32))
    assert c < 1e-4  # |x + 16| stays representable to ~4e-6 A


def test_two_atom_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(20):
        A = rng.normal(0, 5, (2, 3)).astype(np.float32)
        B = rng.normal(0, 5, (2, 3)).astype(np.float32)
        dA = np.linalg.norm(A[0].astype(np.float64) - A[1])
        dB = np.linalg.norm(B[0].astype(np.float64) - B[1])
        assert abs(oracle.crmsd_pair(A, B)[0] - abs(dA - dB) / 2) < 1e-12 * max(dA, dB)


def test_brute_force_rotation_search():
    """4-atom inputs: no rotation on a dense SO(3) sample beats the oracle; local search reaches it."""
    from scipy.optimize import minimize

    rng = np.random.default_rng(6)
    for trial in range(6):
        A = rng.normal(0, 3, (4, 3)).astype(np.float32)
        B = rng.normal(0, 3, (4, 3)).astype(np.float32)
        c, _ = oracle.crmsd_pair(A, B)
        q = rng.standard_normal((200000, 4))
        R = quat_to_R(q)
        a = A.astype(np.float64) - A.astype(np.float64).mean(0)
        b = B.astype(np.float64) - B.astype(np.float64).mean(0)
        vals = np.sqrt(((a[None] - np.einsum("nij,lj->nli", R, b)) ** 2).sum((1, 2)) / 4)
        assert vals.min() >= c - 1e-12
        best = q[np.argmin(vals)]
        f = lambda x: rms_after(quat_to_R(x), A, B)
        res = minimize(f, best, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-14, "maxiter": 20000})
        assert res.fun >= c - 1e-12
        assert res.fun - c < 1e-6


def test_vs_ref_and_pairs_consistent():
    e = E.config0()
    ref = e.coords[7]
    v = oracle.crmsd_vs_ref(e.coords, ref)
    ia = np.arange(e.N)
    p = oracle.crmsd_pairs(e.coords, ia, np.full(e.N, 7))
    assert np.array_equal(v, p)
    assert v[7] < 1e-12


def _loss_rows(X, w, a):
    """Loss terms that depend on model a: sum_b w_ab c_ab."""
    N = X.shape[0]
    others = np.array([b for b in range(N) if b != a])
    c = oracle.crmsd_pairs(X, np.full(len(others), a), others)
    lo = np.minimum(a, others)
    hi = np.maximum(a, others)
    idx = lo * N - lo * (lo + 1) // 2 + (hi - lo - 1)
    return float((w[idx] * c).sum())


def test_allpairs_layout_against_single_pairs():
    """Every entry of the condensed all-versus-all matrix is the single-pair value of the pair its
    index names, idx(a, b) = a N - a (a + 1) / 2 + (b - a - 1) for a < b (the matrix's loop
    bounds and index arithmetic, checked pair by pair on a small ensemble)."""
    e = E.decoy_ensemble(7, 23, 2, (0.5, 6.0), 71)
    X = e.coords
    full = oracle.crmsd_allpairs(X)
    N = X.shape[0]
    assert full.shape == (N * (N - 1) // 2,)
    seen = np.zeros(full.shape, dtype=bool)
    for a in range(N):
        for b in range(a + 1, N):
            k = a * N - a * (a + 1) // 2 + (b - a - 1)
            seen[k] = True
            c, _ = oracle.crmsd_pair(X[a], X[b])
            assert full[k] == c
    assert seen.all()


def test_gradient_matches_finite_differences():
    """Analytic envelope-theorem gradient vs FP64 central differences (exact FP32 steps)."""
    e = E.decoy_ensemble(8, 24, 2, (0.5, 6.0), 77)
    X = e.coords.copy()
    # centre the inputs near the origin so that the FP32 grid is fine
    X = (X - X.mean(axis=1, keepdims=True)).astype(np.float32)
    N = X.shape[0]
    w = E.weights(N * (N - 1) // 2, 78).astype(np.float64)
    g = oracle.crmsd_grad(X, w, eps=1e-6)
    rng = np.random.default_rng(9)
    for _ in range(24):
        a, i, k = rng.integers(N), rng.integers(X.shape[1]), rng.integers(3)
        Xp, Xm = X.copy(), X.copy()
        Xp[a, i, k] = np.float32(X[a, i, k] + 1e-3)
        Xm[a, i, k] = np.float32(X[a, i, k] - 1e-3)
        h = float(Xp[a, i, k]) - float(Xm[a, i, k])
        fd = (_loss_rows(Xp, w, a) - _loss_rows(Xm, w, a)) / h
        assert abs(fd - g[a, i, k]) <= 1e-6 * np.abs(g).max() + 1e-6 * abs(g[a, i, k])


def test_gradient_rows_equal_full_gradient():
    """The per-model gradient entry point returns exactly the rows of the full gradient."""
    e = E.decoy_ensemble(9, 20, 2, (0.5, 5.0), 21)
    N = e.N
    w = E.weights(N * (N - 1) // 2, 22).astype(np.float64)
    g = oracle.crmsd_grad(e.coords, w, eps=1e-6)
    rows = np.array([0, 4, 8])
    gr = oracle.crmsd_grad_rows(e.coords, w, rows, eps=1e-6)
    assert np.abs(gr - g[rows]).max() <= 1e-12 * np.abs(g).max()


def test_gradient_guard_identical_copies():
    """c = 0 exactly (bit-identical copy): the guarded term is finite and zero."""
    e = E.config0()
    X = np.stack([e.coords[0], e.coords[0], e.coords[1]]).astype(np.float32)
    w = np.array([1.0, 0.0, 0.0])  # only the identical pair (0, 1) carries weight
    g = oracle.crmsd_grad(X, w, eps=1e-6)
    assert np.all(np.isfinite(g))
    assert np.abs(g).max() < 1e-6


def test_gradient_symmetry_and_translation_null():
    """Sum over atoms of each model's gradient is zero (translation invariance)."""
    e = E.decoy_ensemble(6, 30, 1, (0.5, 5.0), 11)
    N = e.N
    w = E.weights(N * (N - 1) // 2, 12).astype(np.float64)
    g = oracle.crmsd_grad(e.coords, w)
    assert np.abs(g.sum(axis=1)).max() < 1e-12 * max(1.0, np.abs(g).max()) * 100


MUTANTS = [
    # (description, text in the oracle, replacement, which pin must catch it)
    ("reflection fix dropped", "double d = (det3(U) * det3(V) < 0.0) ? -1.0 : 1.0;", "double d = 1.0;", "mirror"),
    ("no centring", "for (int k = 0; k < 3; ++k) m[k] /= (double)L;", "for (int k = 0; k < 3; ++k) m[k] = 0.0;", "golden"),
    ("rotation transposed", "double rb = R[r][0] * bc[3 * i + 0] + R[r][1] * bc[3 * i + 1] + R[r][2] * bc[3 * i + 2];\n            double e",
     "double rb = R[0][r] * bc[3 * i + 0] + R[1][r] * bc[3 * i + 1] + R[2][r] * bc[3 * i + 2];\n            double e", "eq2"),
    ("1/(L-1) normalisation", "return sqrt(acc / (double)L);", "return sqrt(acc / (double)(L - 1 > 0 ? L - 1 : 1));", "golden"),
]


@pytest.mark.parametrize("mut", MUTANTS, ids=lambda m: m[0])
def test_planted_mistakes_are_caught(mut):
    """Each plausible mistake planted in a copy of the oracle fails one of the pins above."""
    desc, old, new, pin = mut
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, desc
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "mut.c")
        open(p, "w").write(src.replace(old, new))
        so = oracle.build(p, os.path.join(d, "libmut.so"))
        lib = oracle.load(so)
        caught = False
        if pin == "mirror":
            A = E.config0().coords[0]
            B = (A * np.array([1, 1, -1], dtype=np.float32)).astype(np.float32)
            a = A.astype(np.float64) - A.astype(np.float64).mean(0)
            expect = 2.0 * np.sqrt(np.linalg.eigvalsh(a.T @ a)[0] / A.shape[0])
            caught = abs(oracle.crmsd_pair(A, B, lib=lib)[0] - expect) > 1e-6
        elif pin == "golden":
            for _, A, B, val in read_golden():
                if abs(oracle.crmsd_pair(A, B, lib=lib)[0] - val) > 1e-9:
                    caught = True
        elif pin == "eq2":
            e = E.config0()
            for i in range(5):
                if abs(oracle.crmsd_pair(e.coords[i], e.coords[i + 1], lib=lib)[0]
                       - eq2_numpy(e.coords[i], e.coords[i + 1])) > 1e-6:
                    caught = True
        assert caught, f"planted mistake '{desc}' was not caught"

"""Pins for the FP64 dRMSD oracle (eq. 5) against facts fixed by the paper and by mathematics.

No expected value comes from the oracle itself: the hand-derived closed forms in
tests/golden/drmsd_closed_forms.txt, Lagrange's identity (the sum of squared pair
distances equals L^2 times the squared radius of gyration, computed here by centring
instead of by pairs), the invariances of distances (rigid motion, mirror image, a
relabelling of the atoms) and the metric properties of an RMS norm of differences.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1302_4000_b300 import ensembles as E

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "drmsd_closed_forms.txt")


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


@pytest.mark.parametrize("case", read_golden(), ids=lambda c: c[0])
def test_drmsd_closed_forms(case):
    _, A, B, val = case
    assert abs(oracle.drmsd_pair(A, B) - val) <= 1e-12 * max(1.0, val)
    assert abs(oracle.drmsd_pair(B, A) - val) <= 1e-12 * max(1.0, val)


def lagrange_scaled(A):
    """dRMSD(A, 2A) = sqrt(mean over i<j of d_ij^2) = sqrt(2L/(L-1)) R_g (Lagrange's identity)."""
    a = A.astype(np.float64)
    L = a.shape[0]
    rg2 = ((a - a.mean(0)) ** 2).sum() / L
    return np.sqrt(2.0 * L / (L - 1) * rg2)


def test_drmsd_scaling_matches_radius_of_gyration():
    e = E.config0()
    for i in range(4):
        A = e.coords[i]
        B = (2.0 * A).astype(np.float32)  # exact in FP32
        assert abs(oracle.drmsd_pair(A, B) - lagrange_scaled(A)) <= 1e-10 * lagrange_scaled(A)


def test_drmsd_invariances():
    e = E.config0()
    rng = np.random.default_rng(7)
    A, B = e.coords[0], e.coords[1]
    base = oracle.drmsd_pair(A, B)
    # a mirror image has the same distances: exactly zero, and the pair's value is unchanged
    M = (A * np.array([1, -1, 1], dtype=np.float32)).astype(np.float32)
    assert oracle.drmsd_pair(A, M) == 0.0
    assert abs(oracle.drmsd_pair(M, B) - oracle.drmsd_pair(A, B * np.array([1, -1, 1], np.float32))) < 1e-12
    # rigid motion: zero up to the FP32 rounding of the moved coordinates
    Q = E.haar_rotations(1, rng)[0]
    R = (A.astype(np.float64) @ Q.T + np.array([30.0, -20.0, 45.0])).astype(np.float32)
    assert oracle.drmsd_pair(A, R) < 2e-5
    assert abs(oracle.drmsd_pair(R, B) - base) < 2e-5
    # relabelling the atoms of both models permutes the pair list only
    p = rng.permutation(A.shape[0])
    assert abs(oracle.drmsd_pair(A[p], B[p]) - base) <= 1e-12 * base
    assert oracle.drmsd_pair(A, A) == 0.0


def test_drmsd_metric_properties():
    e = E.config0()
    rng = np.random.default_rng(11)
    for _ in range(20):
        i, j, k = rng.choice(e.coords.shape[0], 3, replace=False)
        A, B, C = e.coords[i], e.coords[j], e.coords[k]
        ab, bc, ac = oracle.drmsd_pair(A, B), oracle.drmsd_pair(B, C), oracle.drmsd_pair(A, C)
        assert ab == oracle.drmsd_pair(B, A)
        assert ac <= ab + bc + 1e-12


def test_drmsd_entry_points_agree():
    e = E.config0()
    X = e.coords[:12]
    N = X.shape[0]
    full = oracle.drmsd_allpairs(X)
    ia, ib = np.triu_indices(N, 1)
    assert np.array_equal(full, oracle.drmsd_pairs(X, ia, ib))
    assert full[5] == oracle.drmsd_pair(X[ia[5]], X[ib[5]])
    assert np.array_equal(oracle.drmsd_pairs(X, ib[:7], ia[:7]), full[:7])


def test_drmsd_rejects_bad_arguments():
    A = np.zeros((1, 3), np.float32)
    with pytest.raises(RuntimeError):
        oracle.drmsd_pair(A, A)  # L = 1: eq. 5 needs an atom pair
    X = np.zeros((3, 4, 3), np.float32)
    with pytest.raises(RuntimeError):
        oracle.drmsd_pairs(X, [0], [3])


def test_drmsd_nonfinite_is_nan():
    e = E.config0()
    A = e.coords[0].copy()
    A[3, 1] = np.nan
    assert np.isnan(oracle.drmsd_pair(A, e.coords[1]))


DRMSD_MUTANTS = [
    # (description, text in the oracle, replacement)
    ("squared distances", "d[k++] = sqrt(s);", "d[k++] = s;"),
    ("normalisation without the factor 2", "return sqrt(2.0 * s / ((double)L * (double)(L - 1)));",
     "return sqrt(s / ((double)L * (double)(L - 1)));"),
    ("a dropped neighbour pair", "for (int64_t j = i + 1; j < L; ++j) {", "for (int64_t j = i + 2; j < L; ++j) {"),
    ("one axis dropped", "for (int ax = 0; ax < 3; ++ax) {\n                const double t",
     "for (int ax = 0; ax < 2; ++ax) {\n                const double t"),
    ("normalised by L^2", "return sqrt(2.0 * s / ((double)L * (double)(L - 1)));",
     "return sqrt(2.0 * s / ((double)L * (double)L));"),
]


@pytest.mark.parametrize("mut", DRMSD_MUTANTS, ids=lambda m: m[0])
def test_planted_drmsd_mistakes_are_caught(mut):
    """Each plausible mistake planted in a copy of the dRMSD oracle fails the pins above."""
    desc, old, new = mut
    src = open(oracle._DSRC).read()
    assert src.count(old) == 1, desc
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "mut.c")
        open(p, "w").write(src.replace(old, new))
        lib = oracle.load(oracle.build(p, os.path.join(d, "libmut.so")))
        caught = any(abs(oracle.drmsd_pair(A, B, lib=lib) - val) > 1e-9 * max(1.0, val)
                     for _, A, B, val in read_golden())
        A = E.config0().coords[0]
        caught = caught or abs(oracle.drmsd_pair(A, (2.0 * A).astype(np.float32), lib=lib)
                               - lagrange_scaled(A)) > 1e-9 * lagrange_scaled(A)
        assert caught, f"planted mistake '{desc}' was not caught"

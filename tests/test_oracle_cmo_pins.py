"""Pins for the contact map overlap oracle (eq. 6 and eq. 7) against facts fixed by the paper
and by counting.

No expected value comes from the oracle itself: hand-counted cases
(tests/golden/cmo_closed_forms.txt), a brute-force count with numpy in FP64 (the oracle takes the
contact test in FP64 too; the models are kept clear of the cutoff so that numpy's square root
cannot tip a decision), and the invariances and bounds of the score.
"""
import itertools
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1302_4000_b300 import ensembles as E

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cmo_closed_forms.txt")


def read_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, L, cut, a, b, counts, val, _why = [f.strip() for f in line.split("|", 7)]
        A = np.array([[float(v) for v in r.split()] for r in a.split(";")], dtype=np.float32)
        B = np.array([[float(v) for v in r.split()] for r in b.split(";")], dtype=np.float32)
        assert A.shape == B.shape == (int(L), 3)
        cases.append((name, A, B, float(cut), tuple(int(c) for c in counts.split()), float(val)))
    return cases


@pytest.mark.parametrize("case", read_golden(), ids=lambda c: c[0])
def test_cmo_hand_counted(case):
    _, A, B, cut, counts, val = case
    assert oracle.cmo_counts(A, B, cut) == counts
    assert abs(oracle.cmo_pair(A, B, cut) - val) <= 1e-12 * max(1.0, val)
    assert abs(oracle.cmo_pair(B, A, cut) - val) <= 1e-12 * max(1.0, val)


def brute_counts(A, B, cut):
    """Counts with numpy in FP64 (valid where no distance lies within FP32 rounding of the cutoff)."""
    i, j = np.triu_indices(A.shape[0], 1)
    ca = np.linalg.norm(A[i].astype(np.float64) - A[j], axis=1) < cut
    cb = np.linalg.norm(B[i].astype(np.float64) - B[j], axis=1) < cut
    return int(ca.sum()), int(cb.sum()), int((ca & cb).sum())


def clear_of_cutoff(X, cut, margin=1e-3):
    i, j = np.triu_indices(X.shape[0], 1)
    d = np.linalg.norm(X[i].astype(np.float64) - X[j], axis=1)
    return np.abs(d - cut).min() > margin


def test_cmo_counts_match_brute_force():
    e = E.config0()
    rng = np.random.default_rng(2)
    done = 0
    for _ in range(40):
        a, b = rng.choice(e.coords.shape[0], 2, replace=False)
        A, B = e.coords[a], e.coords[b]
        if not (clear_of_cutoff(A, 8.0) and clear_of_cutoff(B, 8.0)):
            continue
        na, nb, nab = brute_counts(A, B, 8.0)
        assert oracle.cmo_counts(A, B, 8.0) == (na, nb, nab)
        assert abs(oracle.cmo_pair(A, B, 8.0) - 200.0 * nab / (na + nb)) <= 1e-12 * 100
        done += 1
    assert done >= 10


def test_cmo_invariances_and_bounds():
    e = E.config0()
    rng = np.random.default_rng(9)
    A, B = e.coords[3], e.coords[4]
    base = oracle.cmo_pair(A, B, 8.0)
    assert 0.0 <= base <= 100.0
    assert oracle.cmo_pair(A, A, 8.0) == 100.0
    M = (A * np.array([-1, 1, 1], np.float32)).astype(np.float32)
    assert oracle.cmo_pair(A, M, 8.0) == 100.0  # a mirror image has the same map
    p = rng.permutation(A.shape[0])  # relabelling both models' atoms permutes the pair list only
    assert oracle.cmo_pair(A[p], B[p], 8.0) == base
    if clear_of_cutoff(A, 8.0, 1e-2) and clear_of_cutoff(B, 8.0, 1e-2):
        Q = E.haar_rotations(1, rng)[0]
        R = (A.astype(np.float64) @ Q.T + np.array([5.0, -7.0, 11.0])).astype(np.float32)
        assert oracle.cmo_pair(R, B, 8.0) == base
    # contacts only grow with the cutoff
    counts = [oracle.cmo_counts(A, B, c)[0] for c in (4.0, 6.0, 8.0, 12.0, 1e4)]
    assert counts == sorted(counts) and counts[-1] == A.shape[0] * (A.shape[0] - 1) // 2


def test_cmo_entry_points_agree_and_nonfinite():
    e = E.config0()
    X = e.coords[:10].copy()
    X[7, 2, 0] = np.nan
    full = oracle.cmo_allpairs(X, 8.0)
    ia, ib = np.triu_indices(10, 1)
    got = oracle.cmo_pairs(X, ia, ib, 8.0)
    bad = (ia == 7) | (ib == 7)
    assert np.isnan(full[bad]).all() and np.isnan(got[bad]).all()
    assert np.array_equal(full[~bad], got[~bad])
    assert full[3] == oracle.cmo_pair(X[ia[3]], X[ib[3]], 8.0)


CMO_MUTANTS = [
    ("contact test not strict", "c[k++] = d2 < cut2 ? 1 : 0;", "c[k++] = d2 <= cut2 ? 1 : 0;"),
    ("score without the factor 2", "return 100.0 * 2.0 * (double)nab / (double)(na + nb);",
     "return 100.0 * (double)nab / (double)(na + nb);"),
    ("self pairs counted", "for (int64_t j = i + 1; j < L; ++j) {\n            const double dx",
     "for (int64_t j = i; j < L && k < L * (L - 1) / 2; ++j) {\n            const double dx"),
    ("union in the denominator", "return 100.0 * 2.0 * (double)nab / (double)(na + nb);",
     "return 100.0 * 2.0 * (double)nab / (double)(na + nb - nab);"),
]


@pytest.mark.parametrize("mut", CMO_MUTANTS, ids=lambda m: m[0])
def test_planted_cmo_mistakes_are_caught(mut):
    desc, old, new = mut
    src = open(oracle._CSRC).read()
    assert src.count(old) == 1, desc
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "mut.c")
        open(p, "w").write(src.replace(old, new))
        lib = oracle.load(oracle.build(p, os.path.join(d, "libmut.so")))
        caught = any(abs(oracle.cmo_pair(A, B, cut, lib=lib) - val) > 1e-9 * max(1.0, val)
                     for _, A, B, cut, _c, val in read_golden())
        assert caught, f"planted mistake '{desc}' was not caught"

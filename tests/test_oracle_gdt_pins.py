"""Pins for the GDT_TS / TM-score / MaxSub oracle (eq. 3, eq. 4; the paper's superposition
search) against values fixed by the definitions.

A model that equals the reference except for a few displaced atoms has known scores: the search
reaches the identity superposition (from a seed, or by refinement on the atoms within 3.5 A), where
every other atom sits at distance 0 and each displaced one at its displacement. None of the
expected values comes from the oracle.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1302_4000_b300 import ensembles as E


def d0_of(L):
    return max(1.24 * np.cbrt(L - 15.0) - 1.8, 0.5)


def native(L, seed=5):
    return E.native_chain(L, np.random.default_rng(seed)).astype(np.float32)


def displaced(A, atoms, delta, seed=0):
    """A copy of A with each listed atom moved by about delta in its own random direction."""
    rng = np.random.default_rng(seed)
    B = A.copy()
    u = rng.standard_normal((len(atoms), 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    B[atoms] = (A[atoms].astype(np.float64) + delta * u).astype(np.float32)
    return B


def expected(A, B):
    """Scores at the identity superposition, from the FP64 distances |B_i - A_i|."""
    d = np.linalg.norm(B.astype(np.float64) - A.astype(np.float64), axis=1)
    L = len(d)
    c = [np.sum(d < x) for x in (1.0, 2.0, 4.0, 8.0)]
    tm = np.mean(1.0 / (1.0 + (d / d0_of(L)) ** 2))
    ms = np.mean(1.0 / (1.0 + (d / 3.5) ** 2))
    return np.array([sum(c) / (4.0 * L), tm, ms])


def test_identical_and_rigidly_moved_models_score_one():
    A = native(60)
    Q = E.haar_rotations(1, np.random.default_rng(2))[0]
    B = (A.astype(np.float64) @ Q.T + np.array([12.0, -30.0, 7.0])).astype(np.float32)
    got = oracle.gdt_tm_vs_ref(np.stack([A, B]), A)
    assert np.array_equal(got[0], [1.0, 1.0, 1.0])
    assert got[1][0] == 1.0 and abs(got[1][1] - 1.0) < 1e-10 and abs(got[1][2] - 1.0) < 1e-10


@pytest.mark.parametrize("L,delta", [(40, 20.0), (120, 25.0), (16, 20.0), (10, 20.0)])
def test_one_displaced_atom(L, delta):
    """One atom 20 A or more off, too far for any rigid motion that keeps the others within
    8 A to bring it within 8 A: every count is L - 1 and the TM sums take the identity's value.
    Checks d0 = 1.24 (L - 15)^(1/3) - 1.8 (0.5 at L = 16 and L = 10, where the formula falls
    below 0.5), strict counts and GDT_TS as four counts averaged over L."""
    A = native(L)
    B = displaced(A, [L // 3], delta)
    got = oracle.gdt_tm_vs_ref(B[None], A)[0]
    assert np.allclose(got, expected(A, B), rtol=0, atol=1e-9), (got, expected(A, B))
    assert got[0] == (L - 1) / L


def test_refinement_reaches_the_identity():
    """Every third atom 20 A off in a random direction: every seed fragment holds a displaced
    atom, so only the refinement on the atoms within 3.5 A reaches the identity, where the
    other two thirds are exact: GDT_TS = n / L."""
    L = 90
    A = native(L, seed=8)
    moved = list(range(2, L, 3))
    B = displaced(A, moved, 20.0, seed=1)
    got = oracle.gdt_tm_vs_ref(B[None], A)[0]
    assert got[0] == (L - len(moved)) / L
    assert np.allclose(got, expected(A, B), rtol=0, atol=1e-9)


def test_model_and_reference_swap():
    e = E.config0()
    A, B = e.coords[3], e.coords[7]
    ab = oracle.gdt_tm_vs_ref(A[None], B)[0]
    ba = oracle.gdt_tm_vs_ref(B[None], A)[0]
    assert np.allclose(ab, ba, rtol=0, atol=1e-12)
    assert np.all((0.0 <= ab) & (ab <= 1.0))


GDT_MUTANTS = [
    ("d0 constant", "const double d0 = 1.24 * cbrt((double)L - 15.0) - 1.8;",
     "const double d0 = 1.42 * cbrt((double)L - 15.0) - 1.8;"),
    ("no refinement", "if (it == max_refine || ns < 3) break;", "if (1) break;"),
    ("GDT counts not normalised by L", "out[0] = (double)(best_c[0] + best_c[1] + best_c[2] + best_c[3]) / (4.0 * (double)L);",
     "out[0] = (double)(best_c[0] + best_c[1] + best_c[2] + best_c[3]) / 4.0;"),
    ("TM sum over the selected atoms", "if (tm / (double)L > best_tm) best_tm = tm / (double)L;",
     "if (tm / (double)(ns > 0 ? ns : 1) > best_tm) best_tm = tm / (double)(ns > 0 ? ns : 1);"),
    ("MaxSub d0", "const double d0 = tm_d0(L), d0m = 3.5;", "const double d0 = tm_d0(L), d0m = 5.0;"),
]


@pytest.mark.parametrize("mut", GDT_MUTANTS, ids=lambda m: m[0])
def test_planted_gdt_mistakes_are_caught(mut):
    desc, old, new = mut
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, desc
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "mut.c")
        open(p, "w").write(src.replace(old, new))
        lib = oracle.load(oracle.build(p, os.path.join(d, "libmut.so")))
        caught = False
        for L, atoms, seed in ((40, [13], 5), (90, list(range(2, 90, 3)), 8)):
            A = native(L, seed=seed)
            B = displaced(A, atoms, 20.0, seed=0 if L == 40 else 1)
            got = oracle.gdt_tm_vs_ref(B[None], A, lib=lib)[0]
            caught |= not np.allclose(got, expected(A, B), rtol=0, atol=1e-9)
        assert caught, f"planted mistake '{desc}' was not caught"


def drifting_helix(L, c, p):
    """A regular helix (radius 2.3 A, 1.75 rad and 1.5 A rise per atom) as the reference and, as
    the model, the same helix whose atoms past the first third drift along x by c (i - L/3)^p A."""
    t = np.arange(L)
    A = np.stack([2.3 * np.cos(1.75 * t), 2.3 * np.sin(1.75 * t), 1.5 * t], axis=1)
    B = A.copy()
    B[:, 0] += c * np.maximum(0, t - L // 3) ** p
    return A.astype(np.float32), B.astype(np.float32)


def test_stop_rule_four_unchanged_iterations():
    """The refinement stops once the number of selected atoms "does not change in four
    iterations" (four refinements in a row select as many atoms as the one before; at most 20).
    On a helix whose second part drifts away from the reference, the refinements keep moving the
    superposition after the count first repeats or after four refinements, which a search that
    stops there (the shorter reading of the sentence) misses: its GDT_TS is lower. Every
    superposition the shorter search scores is also scored by the longer one, so its scores are
    never higher on any model."""
    for c, short in ((0.33, (1, 20)), (0.42, (4, 4))):
        # drift 0.33: the count repeats once while the atoms still change (a stop at the first
        # repeat misses the last atom); drift 0.42: the count keeps changing past four refinements
        A, B = drifting_helix(32, c, 1.5)
        new = oracle.gdt_tm_vs_ref(B[None], A)[0]
        assert np.array_equal(new, oracle.gdt_tm_vs_ref_rule(B[None], A, 4, 20)[0])
        old = oracle.gdt_tm_vs_ref_rule(B[None], A, 1, 4)[0]
        part = oracle.gdt_tm_vs_ref_rule(B[None], A, *short)[0]
        L = A.shape[0]
        assert round(new[0] * 4 * L) == round(old[0] * 4 * L) + 1  # one more atom within a cutoff
        assert round(new[0] * 4 * L) == round(part[0] * 4 * L) + 1
        assert new[0] > old[0] and new[1] >= old[1] and new[2] >= old[2]
    e = E.config1(N=120)
    Xn = oracle.gdt_tm_vs_ref(e.coords, e.natives[0])
    Xo = oracle.gdt_tm_vs_ref_rule(e.coords, e.natives[0], 1, 4)
    assert np.all(Xn >= Xo - 1e-15)
    # the bound on the refinements counts: with one refinement at most, fewer superpositions
    X1 = oracle.gdt_tm_vs_ref_rule(e.coords, e.natives[0], 4, 1)
    assert np.all(Xn >= X1 - 1e-15)


@pytest.mark.parametrize("mut", [("stop at the first repeated count", "#define GDT_STABLE 4 ", "#define GDT_STABLE 1 "),
                                 ("at most four refinements", "#define GDT_MAX_REFINE 20 ", "#define GDT_MAX_REFINE 4 ")],
                         ids=lambda m: m[0])
def test_planted_stop_rule_mistakes_are_caught(mut):
    """The shorter stop rules, planted in the oracle's default, miss the drifting helix's extra atom."""
    desc, old, new = mut
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, desc
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "mut.c")
        open(p, "w").write(src.replace(old, new))
        lib = oracle.load(oracle.build(p, os.path.join(d, "libmut.so")))
        caught = False
        for c in (0.33, 0.42):
            A, B = drifting_helix(32, c, 1.5)
            L = A.shape[0]
            # the rule's count on this helix: one atom more than the shorter search finds
            want = round(oracle.gdt_tm_vs_ref_rule(B[None], A, 1, 4)[0][0] * 4 * L) + 1
            caught |= round(oracle.gdt_tm_vs_ref(B[None], A, lib=lib)[0][0] * 4 * L) != want
        assert caught, f"planted mistake '{desc}' was not caught"

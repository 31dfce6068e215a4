"""GPU parity: GDT_TS, TM-score and MaxSub against a reference (eq. 3, eq. 4; the paper's
superposition search) through the C-ABI against the oracle.

Both sides take the integer decisions (d < 1, 2, 4, 8 A and the 3.5 A selection) in FP64 on the
same superpositions (fragment seeds, then refinement), so the GDT_TS counts agree exactly (the
score to FP32 rounding, 1e-7); the TM and MaxSub terms are summed in FP32 on the GPU: 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def run(X, ref):
    out = clusco.gdt_tm_vs_ref(torch.from_numpy(X).cuda(), torch.from_numpy(np.ascontiguousarray(ref)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def check(got, ref):
    assert np.all(np.abs(got[:, 0] - ref[:, 0]) <= 1e-7), np.abs(got[:, 0] - ref[:, 0]).max()
    assert np.all(np.abs(got[:, 1:] - ref[:, 1:]) <= 1e-5), np.abs(got[:, 1:] - ref[:, 1:]).max()


@pytest.mark.parametrize("N,L", [(200, 100), (64, 3), (64, 4), (64, 5), (64, 15), (64, 16), (64, 33), (48, 300),
                                 (8, 600)])
def test_scores_match_oracle(N, L):
    """L from the smallest chain (3 atoms: only the whole-chain seed) through lengths where
    4 = L/4 repeats or L/4 < 3 drops, to 300 atoms, and 600 atoms (the staged chain alone below
    the default 48 KB of shared memory, with the kernel's static arrays above it)."""
    e = E.decoy_ensemble(N, L, 2, (0.3, 6.0), seed=13024700 + L)
    ref = e.coords[0]
    got = run(e.coords, ref)
    want = oracle.gdt_tm_vs_ref(e.coords, ref)
    check(got, want)
    assert np.array_equal(got[0], [1.0, 1.0, 1.0])  # the reference itself


def test_largest_supported_chain():
    e = E.decoy_ensemble(12, 1024, 1, (0.5, 4.0), seed=77)
    got = run(e.coords, e.coords[3])
    check(got, oracle.gdt_tm_vs_ref(e.coords, e.coords[3]))


def test_nonfinite_model_and_reference():
    e = E.decoy_ensemble(20, 40, 1, (0.5, 4.0), seed=78)
    X = e.coords.copy()
    X[5, 7, 1] = np.nan
    got = run(X, X[0])
    assert clusco.sync_status() == 6
    assert np.isnan(got[5]).all()
    keep = np.arange(20) != 5
    check(got[keep], oracle.gdt_tm_vs_ref(X[keep], X[0]))
    bad_ref = X[1].copy()
    bad_ref[0, 0] = np.inf
    assert np.isnan(run(X[keep], bad_ref)).all()
    assert clusco.sync_status() == 6


def test_bench_ensemble_against_a_native():
    """The 5,000 x 300 decoy ensemble against one of its natives (the one-versus-reference use
    of the paper), 300 sampled models against the oracle."""
    e = E.config1()
    native = e.natives[0].astype(np.float32)
    got = run(e.coords, native)
    idx = np.random.default_rng(4).choice(e.coords.shape[0], 300, replace=False)
    check(got[idx], oracle.gdt_tm_vs_ref(e.coords[idx], native))


def test_stop_rule_on_drifting_helices():
    """The refinement runs until the selected count has not changed in four iterations: on the
    helices whose second part drifts away (see the oracle's pins), the kernel finds the atom that
    a search stopping at the first repeated count, or after four refinements, misses."""
    t = np.arange(32)
    A = np.stack([2.3 * np.cos(1.75 * t), 2.3 * np.sin(1.75 * t), 1.5 * t], axis=1)
    models = []
    for c in (0.33, 0.42):
        B = A.copy()
        B[:, 0] += c * np.maximum(0, t - 32 // 3) ** 1.5
        models.append(B)
    X = np.stack(models).astype(np.float32)
    A = A.astype(np.float32)
    got = run(X, A)
    want = oracle.gdt_tm_vs_ref(X, A)
    check(got, want)
    # drift 0.33 against a stop at the first repeated count, 0.42 against four refinements at most
    short = np.array([oracle.gdt_tm_vs_ref_rule(X[:1], A, 1, 20)[0, 0], oracle.gdt_tm_vs_ref_rule(X[1:], A, 4, 4)[0, 0]])
    assert np.array_equal(np.round(got[:, 0] * 4 * 32), np.round(short * 4 * 32) + 1)

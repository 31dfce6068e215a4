"""GPU parity: all-versus-all contact map overlap (eq. 6, eq. 7) through the C-ABI against the oracle.

Both forms count contacts exactly (the tensor-core form's FP32 accumulation of 0/1 products stays
below 2^24; the plain form counts bits). The kernels take the contact test in FP32, the oracle in
FP64 (the definition): the two can differ only for atom pairs whose distance lies within FP32
rounding of the cutoff. Where neither model of a pair has such an atom pair the scores agree to the
FP32 rounding of the exact ratio, |S_gpu - S_oracle| <= 2^-21 S; elsewhere the GPU score lies in
the interval those atom pairs allow, and the tests count them. The two forms give bitwise
identical scores.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

from _util import all_pairs, cmo_bounds, condensed_index, contact_band, sample_pairs

pytestmark = pytest.mark.gpu

FORMS = (clusco.FORM_FP8_EXACT, clusco.FORM_FP32_SIMT)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def run(X, cutoff, form):
    out = clusco.cmo_allpairs(torch.from_numpy(X).cuda(), cutoff, form)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(got, ref, X, cutoff, ia=None, ib=None):
    """got, ref over the pairs (ia[k], ib[k]) (every pair a < b when not given)."""
    got = got.astype(np.float64)
    if ia is None:
        ia, ib = all_pairs(X.shape[0])
    band = contact_band(X, cutoff)
    kpair = band[ia] + band[ib]
    strict = kpair == 0
    bad = np.nonzero(strict & ~(np.abs(got - ref) <= 2.0 ** -21 * np.abs(ref)))[0]
    assert bad.size == 0, f"{bad.size} pairs differ, first at {bad[0]}: {got[bad[0]]} vs {ref[bad[0]]}"
    loose = np.nonzero(~strict)[0]
    for q in loose:
        if np.isnan(ref[q]):
            assert np.isnan(got[q])
            continue
        na, nb, nab = oracle.cmo_counts(X[ia[q]], X[ib[q]], cutoff)
        lo, hi = cmo_bounds(na, nb, nab, int(band[ia[q]]), int(band[ib[q]]))
        assert lo * (1 - 2.0 ** -21) <= got[q] <= hi * (1 + 2.0 ** -21), (q, got[q], lo, hi)
    print(f"\ncontact test: {int(band.sum())} atom pairs within FP32 rounding of the cutoff; "
          f"{loose.size} of {got.size} model pairs checked against the interval they allow, "
          f"{int((np.abs(got[loose] - ref[loose]) > 2.0 ** -21 * np.abs(ref[loose])).sum())} of them differ")


@pytest.mark.parametrize("N,L,cutoff", [(200, 100, 8.0), (300, 46, 6.0), (130, 2, 5.0), (257, 181, 8.0),
                                        (513, 64, 12.0)])
def test_cmo_matches_oracle_on_every_pair(N, L, cutoff):
    """Several 128 x 256 tiles with ragged edges (N not a multiple of 256), K from one padded
    block (L = 2) to 16,290 atom pairs, short and long cutoffs."""
    e = E.decoy_ensemble(N, L, 2, (0.5, 8.0), seed=13024600 + N + L)
    ref = oracle.cmo_allpairs(e.coords, cutoff)
    outs = [run(e.coords, cutoff, f) for f in FORMS]
    for got in outs:
        check(got, ref, e.coords, cutoff)
    assert np.array_equal(outs[0], outs[1])


def test_cmo_copies_mirrors_cutoff_edge_and_nonfinite():
    rng = np.random.default_rng(3)
    base = E.decoy_ensemble(60, 80, 1, (0.5, 4.0), seed=21).coords
    # integer coordinates put some distances exactly on the cutoff (strictly below is a contact)
    grid = np.round(base / 2.0).astype(np.float32) * 2.0
    X = np.concatenate([grid, grid[:, ::-1] * np.array([1, 1, -1], np.float32), grid.copy()]).astype(np.float32)
    X[17, 5, 2] = np.nan
    N = X.shape[0]
    ref = oracle.cmo_allpairs(X, 8.0)
    for form in FORMS:
        got = run(X, 8.0, form)
        assert clusco.sync_status() == 6  # CLUSCO_ENONFINITE, read and cleared
        a, b = all_pairs(N)
        badm = (a == 17) | (b == 17)
        assert np.isnan(got[badm]).all()
        check(got[~badm], ref[~badm], X, 8.0, a[~badm], b[~badm])
        for m in range(60):
            if m != 17:
                assert got[condensed_index(m, m + 120, N)] == 100.0  # an exact copy
    # a relabelled mirror (atoms reversed) has the same contacts only up to the relabelling;
    # the plain mirror of model m (no relabelling) scores 100
    Y = np.concatenate([grid[:10], grid[:10] * np.array([-1, 1, 1], np.float32)]).astype(np.float32)
    for form in FORMS:
        got = run(Y, 8.0, form)
        for m in range(10):
            assert got[condensed_index(m, m + 10, 20)] == 100.0


def test_cmo_bench_workload_sampled():
    e = E.config1()
    X = e.coords
    N = X.shape[0]
    outs = [run(X, 8.0, f) for f in FORMS]
    assert np.array_equal(outs[0], outs[1])
    a, b = sample_pairs(N, 4000, seed=5)
    ref = oracle.cmo_pairs(X, a, b, 8.0)
    check(outs[0][condensed_index(a, b, N)], ref, X, 8.0, a, b)


def test_cmo_largest_supported_chain():
    e = E.decoy_ensemble(129, 4096, 2, (0.5, 8.0), seed=33)
    outs = [run(e.coords, 8.0, f) for f in FORMS]
    assert np.array_equal(outs[0], outs[1])
    a, b = sample_pairs(129, 24, seed=9)
    check(outs[0][condensed_index(a, b, 129)], oracle.cmo_pairs(e.coords, a, b, 8.0), e.coords, 8.0, a, b)

"""GPU parity: all-versus-all dRMSD (eq. 5) through the C-ABI against the FP64 oracle.

Tolerances, from the arithmetic of each form:

* BF16_EXACT2: every distance is rounded to the ensemble's 16-bit grid (step q = dmax / 65278,
  dmax the largest intra-model distance of the ensemble) and the Gram matrix of the rounded
  distances is exact, so the result is the exact dRMSD of distances that each moved by at most
  q/2 (plus FP32 rounding of the distance itself, 2^-22 dmax): by the triangle inequality of the
  RMS norm |error| <= q + 2^-21 dmax, plus 2^-22 relative for the final FP32 square root.
* FP32_SIMT: FP32 distances (2^-22 dmax each) differenced directly and summed in FP32 with
  Kahan-compensated 32-term slabs: |error| <= 2^-21 dmax + 1e-6 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

from _util import all_pairs, condensed_index, sample_pairs

pytestmark = pytest.mark.gpu

FORMS = (clusco.FORM_BF16_EXACT2, clusco.FORM_FP32_SIMT)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def max_distance(X, chunk=256):
    """Largest intra-model distance over all finite models (FP64), chunked over models."""
    L = X.shape[1]
    i, j = np.triu_indices(L, 1)
    m = 0.0
    for s in range(0, X.shape[0], chunk):
        x = X[s:s + chunk].astype(np.float64)
        ok = np.isfinite(x).all(axis=(1, 2))
        x = x[ok]
        if len(x):
            m = max(m, float(np.sqrt(((x[:, i] - x[:, j]) ** 2).sum(-1)).max()))
    return m


def bound(form, ref, dmax):
    ref = np.asarray(ref, dtype=np.float64)
    if form == clusco.FORM_BF16_EXACT2:
        return dmax / 65278.0 + dmax * 2.0 ** -21 + 2.0 ** -22 * ref
    return dmax * 2.0 ** -21 + 1e-6 * ref


def run(X, form):
    out = clusco.drmsd_allpairs(torch.from_numpy(X).cuda(), form)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def check(X, form, got, a, b, ref, dmax=None):
    dmax = max_distance(X) if dmax is None else dmax
    err = np.abs(got - ref)
    bnd = bound(form, ref, dmax)
    bad = np.nonzero(~(err <= bnd))[0]
    assert bad.size == 0, (f"form {form}: {bad.size} pairs over the bound, worst "
                           f"{err[bad].max():.3e} at ({a[bad[0]]}, {b[bad[0]]}); bound {bnd[bad[0]]:.3e}")
    return err


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("N,L", [(200, 100), (300, 46), (130, 2), (129, 3), (257, 181)])
def test_drmsd_matches_oracle_on_every_pair(form, N, L):
    """Sizes span several tiles with a ragged last tile (N not a multiple of 128), K from one
    padded block (L = 2, 3) to several 1024-term chunks with a ragged last chunk (L = 46:
    K = 1035; L = 100: K = 4950; L = 181: K = 16290)."""
    e = E.decoy_ensemble(N, L, 2, (0.5, 8.0), seed=13024500 + N + L)
    X = e.coords
    ref = oracle.drmsd_allpairs(X)
    got = run(X, form)
    a, b = all_pairs(N)
    err = check(X, form, got, a, b, ref)
    print(f"\ndRMSD form {form} N={N} L={L}: max |err| {err.max():.2e}, p99 {np.quantile(err, 0.99):.2e}")


@pytest.mark.parametrize("form", FORMS)
def test_drmsd_near_duplicates_copies_and_mirrors(form):
    """Close models (sigma 1e-3 to 0.3 A), exact copies and mirror images: copies and mirrors
    score exactly zero (equal distances round to equal integers), close pairs stay in bound."""
    rng = np.random.default_rng(5)
    base = E.decoy_ensemble(40, 120, 1, (1.0, 6.0), seed=99).coords
    models = [base]
    for s in (1e-3, 1e-2, 0.1, 0.3):
        models.append((base + rng.normal(0.0, s, base.shape)).astype(np.float32))
    models.append(base.copy())
    models.append((base * np.array([1, 1, -1], np.float32)).astype(np.float32))
    X = np.concatenate(models).astype(np.float32)
    N = X.shape[0]
    ref = oracle.drmsd_allpairs(X)
    got = run(X, form)
    a, b = all_pairs(N)
    check(X, form, got, a, b, ref)
    n0 = base.shape[0]
    for m in range(n0):
        for off in (5 * n0, 6 * n0):  # the copy and the mirror of model m
            assert got[condensed_index(m, m + off, N)] == 0.0


@pytest.mark.parametrize("form", FORMS)
def test_drmsd_nonfinite_models(form):
    e = E.decoy_ensemble(150, 50, 1, (0.5, 8.0), seed=7)
    X = e.coords.copy()
    X[17, 3, 1] = np.nan
    X[90, 0, 0] = np.inf
    got = run(X, form)
    assert clusco.sync_status() == 6  # CLUSCO_ENONFINITE, read and cleared
    N = X.shape[0]
    a, b = all_pairs(N)
    badm = (a == 17) | (b == 17) | (a == 90) | (b == 90)
    assert np.isnan(got[badm]).all()
    ref = oracle.drmsd_pairs(X, a[~badm], b[~badm])
    check(X, form, got[~badm], a[~badm], b[~badm], ref)


def test_drmsd_bench_workload_sampled():
    """The 5,000 x 300 decoy ensemble: both forms on the same call shape the benchmark times;
    5,000 sampled pairs and every pair among the first 60 models (close decoys of one native
    included) against the oracle, and the two forms against each other on every pair."""
    e = E.config1()
    X = e.coords
    N = X.shape[0]
    d_exact = run(X, clusco.FORM_BF16_EXACT2)
    d_plain = run(X, clusco.FORM_FP32_SIMT)
    a, b = sample_pairs(N, 5000, seed=3)
    a2, b2 = all_pairs(60)
    a = np.concatenate([a, a2])
    b = np.concatenate([b, b2])
    ref = oracle.drmsd_pairs(X, a, b)
    idx = condensed_index(a, b, N)
    dmax = max_distance(X)
    err_e = check(X, clusco.FORM_BF16_EXACT2, d_exact[idx], a, b, ref, dmax)
    err_p = check(X, clusco.FORM_FP32_SIMT, d_plain[idx], a, b, ref, dmax)
    assert np.all(np.abs(d_exact - d_plain) <= bound(clusco.FORM_BF16_EXACT2, d_plain, dmax)
                  + bound(clusco.FORM_FP32_SIMT, d_plain, dmax))
    print(f"\ndRMSD 5000 x 300: dmax {dmax:.2f} A, q {dmax / 65278:.2e} A; exact max |err| {err_e.max():.2e} "
          f"(p99 {np.quantile(err_e, 0.99):.2e}); plain max |err| {err_p.max():.2e}")


@pytest.mark.parametrize("form", FORMS)
def test_drmsd_largest_supported_chain(form):
    """L = 4096 (the largest supported chain: K = 8,386,560 distances per model, coordinates
    staged in 64 KB of shared memory): sampled pairs against the oracle."""
    e = E.decoy_ensemble(129, 4096, 2, (0.5, 8.0), seed=31)
    X = e.coords
    got = run(X, form)
    a, b = sample_pairs(129, 24, seed=8)
    a = np.concatenate([a, [0, 127]])
    b = np.concatenate([b, [128, 128]])
    ref = oracle.drmsd_pairs(X, a, b)
    check(X, form, got[condensed_index(a, b, 129)], a, b, ref)

"""GPU parity: the CUDA all-pairs and one-vs-reference paths against the FP64 oracle.

Every call goes through the C-ABI (the ctypes binding). Tolerances:

* BF16_EXACT2 (split BF16, exact digit products): 1e-3 A absolute on every pair (the
  tolerance stated for split-BF16 forms); the 16-bit fixed point grid itself moves cRMSD
  by at most about 1e-4 A.
* FP32_SIMT (plain form): 1e-4 A absolute where FP32 accumulation allows it; in general
  |dc| <= dc2 / c with dc2 = 8 sqrt(L) eps32 (G_a + G_b) / L, the bound of FP32
  accumulation of the covariance over L terms (random-walk growth, factor 8 margin)
  pushed through the cancellation in D = R_A^2 + R_B^2 - 2 Sigma.
* TF32 and BF16X3: their input rounding (2^-11 and 2^-17 relative) is not benign on
  near-duplicates; bounds as FP32 with their own unit roundoff.
* INT_SIMT (exact-integer CUDA-core form: 24-bit fixed point, int64 sums, FP64 refinement
  wherever the FP32 bound exceeds 2e-5 A): 1e-4 A absolute on every pair.
* one-vs-reference (24-bit exact integers, FP64 epilogue): 1e-4 A.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

from _util import all_pairs, c_error_bound, condensed_index, gyration_sums, sample_pairs

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def tc_forms():
    return [clusco.FORM_BF16_EXACT2, clusco.FORM_BF16X3, clusco.FORM_TF32]


def forms_available():
    out = [clusco.FORM_FP32_SIMT, clusco.FORM_INT_SIMT]
    X = torch.zeros((4, 8, 3), device="cuda")
    X[:, :, 0] = torch.arange(8, device="cuda")
    for f in tc_forms():
        try:
            clusco.crmsd_allpairs(X, f)
            torch.cuda.synchronize()
            out.append(f)
        except clusco.ClusCoError as e:
            if e.code != 7:
                raise
    return out


def bound_for(form, c_ref, Ga, Gb, L):
    if form == clusco.FORM_BF16_EXACT2:
        return np.full_like(np.asarray(c_ref, dtype=np.float64), 1e-3)
    if form == clusco.FORM_INT_SIMT:
        return np.full_like(np.asarray(c_ref, dtype=np.float64), 1e-4)
    u = {clusco.FORM_FP32_SIMT: EPS32, clusco.FORM_TF32: 2.0 ** -11, clusco.FORM_BF16X3: 2.0 ** -17}[form]
    rel = 8.0 * np.sqrt(L) * u
    return np.maximum(c_error_bound(c_ref, Ga, Gb, L, rel), 1e-4)


def run_allpairs(X, form):
    Xd = torch.from_numpy(X).cuda()
    out = clusco.crmsd_allpairs(Xd, form)
    rc = clusco.sync_status()
    assert rc == 0, clusco.load().clusco_last_error()
    return out.cpu().numpy().astype(np.float64)


def check(form, X, got, ia, ib, ref):
    G = gyration_sums(X)
    L = X.shape[1]
    err = np.abs(got - ref)
    bnd = bound_for(form, ref, G[ia], G[ib], L)
    worst = np.argmax(err / bnd)
    msg = (f"form={form} N={X.shape[0]} L={L}: max|d|={err.max():.3e} p99={np.percentile(err, 99):.3e} "
           f"worst pair ({ia[worst]},{ib[worst]}) c={ref[worst]:.6f} got={got[worst]:.6f} bound={bnd[worst]:.3e}")
    print(msg)
    assert np.all(np.isfinite(got)), msg
    assert np.all(err <= bnd), msg
    return err


@pytest.mark.parametrize("form", [0, 1, 2, 3, 5])
def test_config0_all_pairs(form):
    if form not in forms_available():
        pytest.skip("form not built")
    e = E.config0()
    ref = oracle.crmsd_allpairs(e.coords)
    got = run_allpairs(e.coords, form)
    ia, ib = all_pairs(e.N)
    err = check(form, e.coords, got, ia, ib, ref)
    if form in (clusco.FORM_FP32_SIMT, clusco.FORM_BF16_EXACT2, clusco.FORM_INT_SIMT):
        assert err.max() <= (1e-3 if form == clusco.FORM_BF16_EXACT2 else 1e-4)


@pytest.mark.parametrize("N", [2, 3, 5, 33, 129])
@pytest.mark.parametrize("L", [1, 2, 3, 4, 7, 16, 17, 255])
def test_tiny_shapes_every_pair(N, L):
    e = E.decoy_ensemble(N, L, 1, (0.5, 6.0), 1000 + 7 * N + L)
    ref = oracle.crmsd_allpairs(e.coords)
    ia, ib = all_pairs(N)
    for form in forms_available():
        got = run_allpairs(e.coords, form)
        check(form, e.coords, got, ia, ib, ref)


def test_config1_sampled_at_bench_size():
    """N=5000, L=300 (the bench workload): 20,000 sampled pairs, every form built."""
    e = E.config1()
    ia, ib = sample_pairs(e.N, 20000, 5)
    ref = oracle.crmsd_pairs(e.coords, ia, ib)
    idx = condensed_index(ia, ib, e.N)
    for form in forms_available():
        got = run_allpairs(e.coords, form)[idx]
        check(form, e.coords, got, ia, ib, ref)


def test_panels_equal_one_shot():
    e = E.decoy_ensemble(301, 40, 2, (0.5, 6.0), 31)
    X = torch.from_numpy(e.coords).cuda()
    for form in forms_available():
        full = clusco.crmsd_allpairs(X, form).cpu()
        N = e.N
        pieces = []
        for r0, r1 in [(0, 37), (37, 128), (128, 299), (299, 300)]:
            pieces.append(clusco.crmsd_allpairs_panel(X, r0, r1, form).cpu())
        assert torch.equal(torch.cat(pieces), full)


def test_output_canaries():
    e = E.decoy_ensemble(70, 20, 1, (0.5, 6.0), 8)
    X = torch.from_numpy(e.coords).cuda()
    P = 70 * 69 // 2
    for form in forms_available():
        buf = torch.full((P + 4096,), 12345.0, device="cuda")
        clusco.crmsd_allpairs(X, form, out=buf)
        torch.cuda.synchronize()
        assert torch.all(buf[P:] == 12345.0)
        assert torch.all(buf[:P] != 12345.0)


def test_vs_ref():
    e = E.config1(N=2000)
    ref_model = e.natives[0].astype(np.float32)
    got = clusco.crmsd_vs_ref(torch.from_numpy(e.coords).cuda(), torch.from_numpy(ref_model).cuda()).cpu().numpy()
    want = oracle.crmsd_vs_ref(e.coords, ref_model)
    assert clusco.sync_status() == 0
    err = np.abs(got - want)
    print(f"vs_ref max|d|={err.max():.3e}")
    assert err.max() <= 1e-4


def test_vs_ref_tiny():
    for L in (1, 2, 3, 5, 64, 1000):
        e = E.decoy_ensemble(17, L, 1, (0.1, 4.0), 90 + L)
        got = clusco.crmsd_vs_ref(torch.from_numpy(e.coords).cuda(), torch.from_numpy(e.coords[3]).cuda()).cpu().numpy()
        want = oracle.crmsd_vs_ref(e.coords, e.coords[3])
        assert np.abs(got - want).max() <= 1e-4, L


def test_nonfinite_inputs_flagged():
    e = E.decoy_ensemble(50, 30, 1, (0.5, 6.0), 12)
    X = e.coords.copy()
    X[7, 3, 1] = np.nan
    Xd = torch.from_numpy(X).cuda()
    for form in forms_available():
        out = clusco.crmsd_allpairs(Xd, form).cpu().numpy()
        assert clusco.sync_status() == 6
        ia, ib = all_pairs(50)
        bad = (ia == 7) | (ib == 7)
        assert np.all(np.isnan(out[bad]))
        assert np.all(np.isfinite(out[~bad]))
    assert clusco.sync_status() == 0


def test_refinement_of_flagged_pairs_in_panels():
    """Near-duplicate models (sigma 0.01-0.1 A): nearly every pair fails the FP32 bound and is
    recomputed by the refinement kernel from the exact fixed-point coordinates. The one-shot
    matrix is held to the exact-digit tolerance against the oracle, and row panels whose pair
    ranges start inside a 32-pair mask word (and a pair count that is not a multiple of 32)
    reproduce it bit for bit."""
    if clusco.FORM_BF16_EXACT2 not in forms_available():
        pytest.skip("exact-digit form unavailable")
    e = E.decoy_ensemble(151, 64, 2, (0.01, 0.1), 77)
    N = e.N
    assert (N * (N - 1) // 2) % 32 != 0
    X = torch.from_numpy(e.coords).cuda()
    full = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    ia, ib = np.triu_indices(N, 1)
    ref = oracle.crmsd_pairs(e.coords, ia, ib)
    err = np.abs(full.double().cpu().numpy() - ref)
    print(f"near-duplicate ensemble: c in [{ref.min():.3f}, {ref.max():.3f}] A, max |d| {err.max():.2e}")
    assert err.max() <= 1e-3
    pieces = [clusco.crmsd_allpairs_panel(X, r0, r1, clusco.FORM_BF16_EXACT2).cpu()
              for r0, r1 in [(0, 1), (1, 37), (37, 101), (101, 149), (149, 150)]]
    assert torch.equal(torch.cat(pieces), full.cpu())


def _sorted_list(idx, vals):
    order = torch.argsort(idx)
    return idx[order], vals[order]


def test_pairs_below_threshold_equal_the_matrix_and_the_oracle():
    """Threshold mode returns exactly the dense matrix's entries below tau (same form, bit for
    bit, in any order), for tau = 0, 3.2 A, the median and +inf, through the retry path of a
    too small first capacity; against the oracle, the exact-digit list holds every pair below
    tau - 1e-3 A and none at or above tau + 1e-3 A (the form's tolerance band)."""
    e = E.config0()
    N = e.N
    X = torch.from_numpy(e.coords).cuda()
    ia, ib = all_pairs(N)
    ref = oracle.crmsd_pairs(e.coords, ia, ib)
    for form in forms_available():
        full = clusco.crmsd_allpairs(X, form)
        for tau in (0.0, 3.2, float(np.median(ref)), float("inf")):
            idx, vals = _sorted_list(*clusco.crmsd_pairs_below(X, tau, form, capacity=64))
            assert clusco.sync_status() == 0
            want = torch.nonzero(full < tau).squeeze(1)
            assert torch.equal(idx, want), (form, tau)
            assert torch.equal(vals, full[want]), (form, tau)
            if form == clusco.FORM_BF16_EXACT2:
                got = np.zeros(len(ref), dtype=bool)
                got[idx.cpu().numpy()] = True
                assert got[ref < tau - 1e-3].all(), tau
                assert not got[ref >= tau + 1e-3].any(), tau
    a, b = clusco.condensed_pairs(idx, N)
    assert torch.all(a < b) and torch.all(b < N)


def test_pairs_below_threshold_skip_nonfinite_models():
    e = E.decoy_ensemble(60, 30, 1, (0.5, 6.0), 19)
    C = e.coords.copy()
    C[11, 4, 2] = np.nan
    X = torch.from_numpy(C).cuda()
    N = e.N
    for form in forms_available():
        idx, vals = clusco.crmsd_pairs_below(X, float("inf"), form)
        clusco.sync_status()  # the non-finite model sets the status word; it is cleared here
        a, b = clusco.condensed_pairs(idx, N)
        assert idx.numel() == (N - 1) * (N - 2) // 2, form  # every pair without model 11
        assert not torch.any((a == 11) | (b == 11)) and torch.all(torch.isfinite(vals))


def test_pairs_below_threshold_bench_workload():
    """The 5,000 x 300 bench ensemble at the paper's 3.2 A cutoff in the exact-digit form: the
    list equals the dense matrix below the cutoff, bit for bit; times both calls."""
    if clusco.FORM_BF16_EXACT2 not in forms_available():
        pytest.skip("exact-digit form unavailable")
    e = E.config1()
    X = torch.from_numpy(e.coords).cuda()
    N, L = e.N, e.L
    P = N * (N - 1) // 2
    full = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    idx, vals = _sorted_list(*clusco.crmsd_pairs_below(X, 3.2, clusco.FORM_BF16_EXACT2, capacity=P))
    want = torch.nonzero(full < 3.2).squeeze(1)
    assert torch.equal(idx, want) and torch.equal(vals, full[want])
    ws = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N, L), dtype=torch.uint8, device="cuda")
    lst = torch.empty(idx.numel() + 1024, dtype=torch.int64, device="cuda")
    val = torch.empty(idx.numel() + 1024, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    lib = clusco.load()
    st = torch.cuda.current_stream().cuda_stream

    def dense():
        clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2, out=full, workspace=ws)

    def below():
        assert lib.clusco_crmsd_allpairs_below(X.data_ptr(), N, L, 3.2, lst.data_ptr(), val.data_ptr(), lst.numel(),
                                               cnt.data_ptr(), clusco.FORM_BF16_EXACT2, ws.data_ptr(), ws.numel(),
                                               st) == 0

    t = {}
    for name, fn in (("dense", dense), ("below", below)):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(10):
            fn()
        b.record()
        torch.cuda.synchronize()
        t[name] = a.elapsed_time(b) / 10
    assert int(cnt.item()) == idx.numel()
    print(f"\n3.2 A cutoff at 5000 x 300: {idx.numel()} of {P} pairs kept; dense {t['dense']:.3f} ms, "
          f"threshold {t['below']:.3f} ms")

"""GPU parity at the full sizes of the precision and large configurations (sampled outputs).

* Precision ensemble (20,000 x 150, half of it near-duplicate clusters, sigma 0.02-0.5 A):
  every form; all 95,000 intra-cluster pairs plus 20,000 random pairs against the FP64
  oracle; max and p99 |d| printed per form and pair class. Exact-digit BF16 must stay within
  1e-3 A on every sampled pair, the exact-integer CUDA-core form within 1e-4 A; the other
  forms within their accumulation bounds.
* Large ensemble (50,000 x 1,000, 1.25e9 pairs, 5 GB condensed output kept on the device):
  exact-digit BF16 on 20,000 sampled pairs; a row panel equals the same slice of the full
  matrix; the plain form on one panel.
* Large adjoint (8,192 x 500; above the tensor-core adjoint's 320-atom limit, so the CUDA-core
  path): gradient rows of sampled models against the oracle's rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

from _util import c_error_bound, condensed_index, gyration_sums, sample_pairs

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def gather(out, ia, ib, N):
    idx = torch.from_numpy(condensed_index(ia, ib, N)).cuda()
    return out[idx].double().cpu().numpy()


def bound(form, ref, Ga, Gb, L):
    if form == clusco.FORM_BF16_EXACT2:
        return np.full_like(ref, 1e-3)
    if form == clusco.FORM_INT_SIMT:
        return np.full_like(ref, 1e-4)
    u = {clusco.FORM_FP32_SIMT: EPS32, clusco.FORM_TF32: 2.0 ** -11, clusco.FORM_BF16X3: 2.0 ** -17}[form]
    return np.maximum(c_error_bound(ref, Ga, Gb, L, 8.0 * np.sqrt(L) * u), 1e-4)


def test_precision_ensemble_every_form():
    e = E.config2()
    N, L = e.N, e.L
    cl = e.extra["cluster"]
    members = {}
    for i, c in enumerate(cl):
        if c >= 0:
            members.setdefault(int(c), []).append(i)
    da, db = [], []
    for m in members.values():
        m = sorted(m)
        for x in range(len(m)):
            for y in range(x + 1, len(m)):
                da.append(m[x])
                db.append(m[y])
    da, db = np.array(da, dtype=np.int64), np.array(db, dtype=np.int64)
    ra, rb = sample_pairs(N, 20000, 202)
    ia, ib = np.concatenate([da, ra]), np.concatenate([db, rb])
    ref = oracle.crmsd_pairs(e.coords, ia, ib)
    G = gyration_sums(e.coords)
    X = torch.from_numpy(e.coords).cuda()
    nd = len(da)
    print(f"\nprecision ensemble N={N} L={L}: {nd} intra-cluster pairs (c {ref[:nd].min():.3f}-{ref[:nd].max():.3f} A), "
          f"{len(ra)} random pairs")
    for form in (clusco.FORM_BF16_EXACT2, clusco.FORM_BF16X3, clusco.FORM_TF32, clusco.FORM_FP32_SIMT,
                 clusco.FORM_INT_SIMT):
        out = clusco.crmsd_allpairs(X, form)
        assert clusco.sync_status() == 0
        got = gather(out, ia, ib, N)
        del out
        torch.cuda.empty_cache()
        err = np.abs(got - ref)
        print(f"  form {form}: near-dup max {err[:nd].max():.3e} p99 {np.percentile(err[:nd], 99):.3e} | "
              f"random max {err[nd:].max():.3e} p99 {np.percentile(err[nd:], 99):.3e}")
        assert np.all(np.isfinite(got))
        assert np.all(err <= bound(form, ref, G[ia], G[ib], L))


def test_large_forward_sampled_and_panel():
    e = E.config4()
    N, L = e.N, e.L
    X = torch.from_numpy(e.coords).cuda()
    out = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    ia, ib = sample_pairs(N, 20000, 404)
    # include the last pair and pairs of the last rows (the largest condensed indices)
    ia = np.concatenate([ia, [N - 2, N - 3, 0]])
    ib = np.concatenate([ib, [N - 1, N - 1, N - 1]])
    ref = oracle.crmsd_pairs(e.coords, ia, ib)
    got = gather(out, ia, ib, N)
    err = np.abs(got - ref)
    print(f"\nlarge ensemble N={N} L={L}: exact-digit max {err.max():.3e} p99 {np.percentile(err, 99):.3e}")
    assert err.max() <= 1e-3
    # a row panel equals the same slice of the one-shot matrix
    r0, r1 = 24990, 25007
    panel = clusco.crmsd_allpairs_panel(X, r0, r1, clusco.FORM_BF16_EXACT2)
    s0 = int(condensed_index(r0, r0 + 1, N))
    assert torch.equal(panel, out[s0:s0 + panel.numel()])
    del out
    torch.cuda.empty_cache()
    # the plain form on one panel (its full matrix would take tens of seconds)
    pp = clusco.crmsd_allpairs_panel(X, 0, 8, clusco.FORM_FP32_SIMT).double().cpu().numpy()
    pa = np.concatenate([np.full(N - 1 - a, a) for a in range(8)])
    pb = np.concatenate([np.arange(a + 1, N) for a in range(8)])
    sel = np.random.default_rng(5).choice(len(pa), 4000, replace=False)
    refp = oracle.crmsd_pairs(e.coords, pa[sel], pb[sel])
    G = gyration_sums(e.coords)
    assert np.all(np.abs(pp[sel] - refp) <= bound(clusco.FORM_FP32_SIMT, refp, G[pa[sel]], G[pb[sel]], L))


def test_large_backward_rows():
    e = E.config4(N=8192, L=500)
    N, L = e.N, e.L
    w = E.weights(N * (N - 1) // 2, 505)
    X = torch.from_numpy(e.coords).cuda()
    c = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward(X, torch.from_numpy(w).cuda(), c, 1e-6, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    rows = np.array([0, 1, 4095, N - 1])
    gref = oracle.crmsd_grad_rows(e.coords, w.astype(np.float64), rows, 1e-6)
    gg = g[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    rel = np.linalg.norm((gg - gref).reshape(len(rows), -1), axis=1) / np.linalg.norm(gref.reshape(len(rows), -1), axis=1)
    print(f"\nlarge adjoint N={N} L={L}: per-model rel err {rel}")
    assert rel.max() <= 1e-3

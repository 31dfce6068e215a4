"""GPU parity of the stored-rotation path: the forward's per-pair rotations and the adjoint
that contracts from them (no covariance recomputation).

Rotations: R_ab is unique except at degenerate covariances, so each stored R is checked for
what is unique (orthogonality, det +1, and that it attains the oracle's cRMSD when applied to
the FP32 coordinates in FP64) and, where the optimum is well separated, element by element
against the oracle's Kabsch rotation. Gradients: the same tolerance as the recompute path
(per model 1e-3 relative, per coordinate 1e-3 (|g_ref| + rms)).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

from _util import all_pairs, condensed_index, sample_pairs

pytestmark = pytest.mark.gpu

TC_FORMS = (clusco.FORM_BF16_EXACT2, clusco.FORM_BF16X3, clusco.FORM_TF32)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def applied_crmsd(X, ia, ib, R):
    """(sqrt(mean |a_i - R b_i|^2), R_A^2 + R_B^2) over centred FP32 coordinates, in FP64."""
    A = X[ia].astype(np.float64)
    B = X[ib].astype(np.float64)
    A -= A.mean(axis=1, keepdims=True)
    B -= B.mean(axis=1, keepdims=True)
    res = A - np.einsum("pij,plj->pli", R, B)
    L = X.shape[1]
    return np.sqrt((res ** 2).sum(axis=(1, 2)) / L), ((A ** 2).sum(axis=(1, 2)) + (B ** 2).sum(axis=(1, 2))) / L


def check_rotations(X, ia, ib, R, c_ref, what):
    R = R.astype(np.float64)
    orth = np.abs(np.einsum("pki,pkj->pij", R, R) - np.eye(3)).max(axis=(1, 2))
    det = np.linalg.det(R)
    c_app, g2 = applied_crmsd(X, ia, ib, R)
    # the applied rotation attains the optimum: c_app^2 - c_ref^2 is second order in the
    # rotation's angle error and first order in its departure from orthogonality (which
    # scales R_A^2 + R_B^2), so the bound is relative to that scale
    gap = np.abs(c_app ** 2 - c_ref ** 2) / g2
    print(f"{what}: max |R^T R - I| {orth.max():.2e}, det in [{det.min():.6f}, {det.max():.6f}], "
          f"max |c^2 gap| / (R_A^2 + R_B^2) {gap.max():.2e}")
    assert orth.max() <= 2e-5, what
    assert np.all(np.abs(det - 1.0) <= 3e-5), what
    assert np.all(gap <= 2e-5), what


def test_rotations_every_pair_config0():
    e = E.config0()
    N = e.N
    X = torch.from_numpy(e.coords).cuda()
    ia, ib = all_pairs(N)
    c_ref = oracle.crmsd_pairs(e.coords, ia, ib)
    plain = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    for form in TC_FORMS:
        out, rot = clusco.crmsd_allpairs_rot(X, form)
        assert clusco.sync_status() == 0
        if form == clusco.FORM_BF16_EXACT2:
            # the rotation variant is a separate compiled kernel: the same arithmetic up to the
            # compiler's contraction choices, so the two agree within twice the FP32 fast
            # path's accepted error (5e-4 A; larger errors are refined in FP64 by both)
            d = (out - plain).abs().max().item()
            assert d <= 1e-3, d
            assert np.abs(out.double().cpu().numpy() - c_ref).max() <= 1e-3
        assert torch.all(rot[:, 9:] == 0)
        R = clusco.rotations_view(rot).double().cpu().numpy()
        check_rotations(e.coords, ia, ib, R, c_ref, f"config0 form {form}")
    # element-wise against the oracle's Kabsch rotation where the optimum is well separated
    R = clusco.rotations_view(clusco.crmsd_allpairs_rot(X, clusco.FORM_BF16_EXACT2)[1]).double().cpu().numpy()
    sel = np.random.default_rng(1).choice(len(ia), 400, replace=False)
    worst = 0.0
    for k in sel:
        A, B = e.coords[ia[k]], e.coords[ib[k]]
        Am = A.astype(np.float64) - A.astype(np.float64).mean(0)
        Bm = B.astype(np.float64) - B.astype(np.float64).mean(0)
        s = np.linalg.svd(Am.T @ Bm, compute_uv=False)
        d = np.sign(np.linalg.det(Am.T @ Bm))
        if (s[1] + d * s[2]) < 0.05 * s[0]:
            continue
        worst = max(worst, np.abs(R[k] - oracle.crmsd_pair(A, B)[1]).max())
    print(f"element-wise max |R - R_oracle| {worst:.2e}")
    assert worst <= 1e-4


def test_rotations_bench_sample():
    e = E.config1()
    N = e.N
    X = torch.from_numpy(e.coords).cuda()
    out, rot = clusco.crmsd_allpairs_rot(X, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    ia, ib = sample_pairs(N, 5000, 11)
    idx = torch.from_numpy(condensed_index(ia, ib, N)).cuda()
    R = clusco.rotations_view(rot)[idx].double().cpu().numpy()
    check_rotations(e.coords, ia, ib, R, oracle.crmsd_pairs(e.coords, ia, ib), "5000 x 300 sample")


@pytest.mark.parametrize("N,L", [(2, 1), (3, 2), (5, 3), (33, 16), (129, 255), (64, 500)])
def test_backward_rot_small_shapes(N, L):
    e = E.decoy_ensemble(N, L, 1, (0.5, 6.0), 1000 + N + L)
    w = E.weights(N * (N - 1) // 2, 17 + N)
    X = torch.from_numpy(e.coords).cuda()
    out, rot = clusco.crmsd_allpairs_rot(X, clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward_rot(X, torch.from_numpy(w).cuda(), out, rot, 1e-6)
    assert clusco.sync_status() == 0
    gref = oracle.crmsd_grad(e.coords, w.astype(np.float64), 1e-6)
    gg = g.double().cpu().numpy()
    na = np.linalg.norm((gg - gref).reshape(N, -1), axis=1)
    nr = np.linalg.norm(gref.reshape(N, -1), axis=1)
    rel = na / np.maximum(nr, 1e-300)
    print(f"N={N} L={L}: max per-model rel err {rel.max():.3e}")
    assert rel.max() <= 1e-3


def test_backward_rot_config3_vs_oracle_and_recompute():
    e, w = E.config3()
    N = e.N
    eps = 1e-6
    X = torch.from_numpy(e.coords).cuda()
    wd = torch.from_numpy(w).cuda()
    out, rot = clusco.crmsd_allpairs_rot(X, clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward_rot(X, wd, out, rot, eps)
    g2 = clusco.crmsd_allpairs_backward(X, wd, out, eps, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    gref = oracle.crmsd_grad(e.coords, w.astype(np.float64), eps)
    gg = g.double().cpu().numpy()
    na = np.linalg.norm((gg - gref).reshape(N, -1), axis=1)
    nr = np.linalg.norm(gref.reshape(N, -1), axis=1)
    rel = na / nr
    rms = np.sqrt((gref.reshape(N, -1) ** 2).mean(axis=1))[:, None, None]
    coord = np.abs(gg - gref) <= 1e-3 * (np.abs(gref) + rms)
    d = ((g - g2).reshape(N, -1).norm(dim=1) / g2.reshape(N, -1).norm(dim=1)).max().item()
    print(f"config3 stored rotations: max per-model rel err {rel.max():.3e}, coords ok {coord.mean():.6f}, "
          f"vs recompute path {d:.2e}")
    assert rel.max() <= 1e-3
    assert coord.all()
    assert d <= 5e-4


def test_autograd_uses_stored_rotations():
    e, w = E.config3()
    N = 300
    X = torch.from_numpy(e.coords[:N]).cuda().requires_grad_(True)
    wt = torch.from_numpy(w[: N * (N - 1) // 2]).cuda()
    loss = (wt * clusco.crmsd_matrix(X, clusco.FORM_BF16_EXACT2, 1e-6, store_rotations=True)).sum()
    loss.backward()
    out, rot = clusco.crmsd_allpairs_rot(X.detach(), clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward_rot(X.detach(), wt, out, rot, 1e-6)
    torch.cuda.synchronize()
    d = (X.grad - g).reshape(N, -1).norm(dim=1) / g.reshape(N, -1).norm(dim=1)
    assert float(d.max()) <= 1e-5


def test_rot_argument_errors():
    X = torch.zeros((4, 600, 3), device="cuda")
    X[:, :, 0] = torch.arange(600, device="cuda")
    P = 6
    with pytest.raises(clusco.ClusCoError):  # the plain form produces no rotations
        clusco.crmsd_allpairs_rot(X, clusco.FORM_FP32_SIMT)
    out = torch.zeros(P, device="cuda")
    rot = torch.zeros((P, clusco.ROT_STRIDE), device="cuda")
    with pytest.raises(clusco.ClusCoError):  # above the 512 atoms of the stored-rotation adjoint
        clusco.crmsd_allpairs_backward_rot(X, torch.ones(P, device="cuda"), out, rot, 1e-6)


@pytest.mark.parametrize("which", ["bench 5000 x 300", "large 8192 x 500"])
def test_backward_rot_full_size_rows(which):
    """The bench's workload (and the large forward+backward size) in the launch configuration
    the bench times: sampled rows of the gradient against the oracle's per-row FP64 gradient."""
    if which.startswith("bench"):
        e = E.config1()
        w = E.weights(e.N * (e.N - 1) // 2, E.SEED_BASE + 101)
    else:
        e = E.config4(N=8192, L=500)
        w = E.weights(e.N * (e.N - 1) // 2, 505)
    N = e.N
    X = torch.from_numpy(e.coords).cuda()
    out, rot = clusco.crmsd_allpairs_rot(X, clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward_rot(X, torch.from_numpy(w).cuda(), out, rot, 1e-6)
    assert clusco.sync_status() == 0
    rows = np.unique(np.concatenate([[0, 1, 39, 40, N // 2, N - 1],
                                     np.random.default_rng(5).integers(0, N, 3)]))
    gref = oracle.crmsd_grad_rows(e.coords, w.astype(np.float64), rows, 1e-6)
    gg = g[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    rel = np.linalg.norm((gg - gref).reshape(len(rows), -1), axis=1) / np.linalg.norm(gref.reshape(len(rows), -1), axis=1)
    rms = np.sqrt((gref.reshape(len(rows), -1) ** 2).mean(axis=1))[:, None, None]
    coord = np.abs(gg - gref) <= 1e-3 * (np.abs(gref) + rms)
    print(f"\n{which}: per-model rel err {rel.max():.3e}, coords ok {coord.mean():.6f}")
    assert rel.max() <= 1e-3
    assert coord.all()


@pytest.mark.parametrize("N,L,form", [(2, 1, clusco.FORM_BF16_EXACT2), (129, 255, clusco.FORM_BF16_EXACT2),
                                      (300, 100, clusco.FORM_TF32), (5000, 300, clusco.FORM_BF16_EXACT2)])
def test_fused_step_equals_the_two_calls(N, L, form):
    """clusco_crmsd_allpairs_step_rot runs the same kernels on the same inputs as the forward and
    adjoint calls made in turn (only the adjoint's pre-pass moves to a side stream): the matrix
    and the rotations are bitwise the same; the gradient is the same up to the order of its
    atomically accumulated FP32 terms (the near-duplicate pairs' direct terms and the per-model
    coefficient sums), which varies from run to run, so it is compared per model to 1e-5 of its
    norm (the accuracy bar against the oracle is 1e-3); the small shapes also go against the
    oracle's gradient."""
    e = E.config1(N=N, L=L) if N == 5000 else E.decoy_ensemble(N, L, 2, (0.5, 6.0), 2000 + N + L)
    w = torch.from_numpy(E.weights(N * (N - 1) // 2, 29 + N)).cuda()
    X = torch.from_numpy(e.coords).cuda()
    out, rot = clusco.crmsd_allpairs_rot(X, form)
    g = clusco.crmsd_allpairs_backward_rot(X, w, out, rot, 1e-6)
    out2, rot2, g2 = clusco.crmsd_allpairs_step_rot(X, w, form, 1e-6)
    assert clusco.sync_status() == 0

    def same_grad(ga, gb):
        d = torch.linalg.vector_norm((ga - gb).double().reshape(N, -1), dim=1)
        nrm = torch.linalg.vector_norm(ga.double().reshape(N, -1), dim=1)
        return bool((d <= 1e-5 * nrm.clamp_min(1e-30)).all())
    assert torch.equal(out, out2) and torch.equal(rot, rot2) and same_grad(g, g2)
    # on another stream, with a caller's workspace and output buffers
    s = torch.cuda.Stream()
    ws = torch.empty(clusco.workspace_bytes(clusco.OP_STEP_ROT, N, L, form), dtype=torch.uint8, device="cuda")
    o3, r3, g3 = torch.full_like(out, -1.0), torch.full_like(rot, -1.0), torch.full_like(g, -1.0)
    s.wait_stream(torch.cuda.current_stream())
    clusco.crmsd_allpairs_step_rot(X, w, form, 1e-6, out=o3, rot=r3, grad_coords=g3, workspace=ws, stream=s)
    assert clusco.sync_status(s) == 0
    assert torch.equal(out, o3) and torch.equal(rot, r3) and same_grad(g, g3)
    if N <= 300:
        gref = oracle.crmsd_grad(e.coords, w.double().cpu().numpy(), 1e-6)
        gg = g2.double().cpu().numpy()
        rel = (np.linalg.norm((gg - gref).reshape(N, -1), axis=1)
               / np.maximum(np.linalg.norm(gref.reshape(N, -1), axis=1), 1e-300))
        assert rel.max() <= 1e-3


def test_fused_step_argument_errors():
    X = torch.zeros((4, 600, 3), device="cuda")
    w = torch.ones(6, device="cuda")
    with pytest.raises(clusco.ClusCoError):  # the plain form produces no rotations
        clusco.crmsd_allpairs_step_rot(X[:, :300].contiguous(), w, clusco.FORM_FP32_SIMT)
    with pytest.raises(clusco.ClusCoError):  # above the 512 atoms of the stored-rotation adjoint
        clusco.crmsd_allpairs_step_rot(X, w, clusco.FORM_BF16_EXACT2)
    assert clusco.workspace_bytes(clusco.OP_STEP_ROT, 4, 600, clusco.FORM_BF16_EXACT2) == 0
    assert clusco.workspace_bytes(clusco.OP_STEP_ROT, 4, 300, clusco.FORM_FP32_SIMT) == 0

"""GPU parity of the tensor-core adjoint that recomputes every pair's rotation (nothing stored
by the forward), against the oracle's FP64 analytic gradient, for L from 1 to 1,000 atoms.

The atoms of a 128-row tile's gradient sum are split over C = ceil(Lp / 384) CTAs; on a B300
those CTAs form a thread-block cluster and share the covariances and rotations through
distributed shared memory. With CLUSCO_BACKWARD_CLUSTERS=0 each chunk CTA recomputes them
instead: both paths are checked, and against each other.

Tolerance (the stated ``<= 1e-3 relative`` for gradients, read per model):
    ||g_a - g_a^oracle||_2 <= 1e-3 ||g_a^oracle||_2 for every model a,
and per coordinate |dg_ai| <= 1e-3 (|g_ai^oracle| + rms(g_a^oracle)).
"""
import os

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


@pytest.fixture(params=["clusters", "no clusters"])
def mode(request, monkeypatch):
    if request.param == "no clusters":
        monkeypatch.setenv("CLUSCO_BACKWARD_CLUSTERS", "0")
    else:
        monkeypatch.delenv("CLUSCO_BACKWARD_CLUSTERS", raising=False)
    return request.param


def grad_tc(X, w, eps, c=None, status=0):
    Xd = torch.from_numpy(X).cuda()
    wd = torch.from_numpy(w).cuda()
    if c is None:
        c = clusco.crmsd_allpairs(Xd, clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward(Xd, wd, c, eps, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == status, clusco.load().clusco_last_error()
    return g.double().cpu().numpy(), c


def compare(g, gref, what, rel_tol=1e-3):
    n = g.shape[0]
    na = np.linalg.norm((g - gref).reshape(n, -1), axis=1)
    nr = np.linalg.norm(gref.reshape(n, -1), axis=1)
    rel = na / np.maximum(nr, 1e-300)
    rms = np.sqrt((gref.reshape(n, -1) ** 2).mean(axis=1))[:, None, None]
    coord = np.abs(g - gref) <= 1e-3 * (np.abs(gref) + rms)
    print(f"{what}: max per-model rel err {rel.max():.3e} (model {np.argmax(rel)}), coords ok {coord.mean():.6f}")
    assert rel.max() <= rel_tol, what
    assert coord.all(), what
    return rel.max()


# L covers one 64-atom K block, ragged K blocks, one and several 128-atom accumulator blocks, and
# one, two and three chunk CTAs (L 300 -> 1 chunk, 500 -> 2, 700 and 1000 -> 2 and 3)
@pytest.mark.parametrize("N,L", [(2, 1), (3, 2), (5, 3), (33, 16), (129, 255), (41, 300), (64, 500),
                                 (81, 700), (45, 1000)])
def test_small_shapes_every_coordinate(N, L, mode):
    e = E.decoy_ensemble(N, L, 1, (0.5, 6.0), 2000 + N + L)
    w = E.weights(N * (N - 1) // 2, 31 + N)
    g, _ = grad_tc(e.coords, w, 1e-6)
    gref = oracle.crmsd_grad(e.coords, w.astype(np.float64), 1e-6)
    compare(g, gref, f"N={N} L={L} {mode}")


@pytest.mark.parametrize("eps", [1e-6, 1e-3])
def test_config3_direct_vs_oracle(eps, mode):
    """The differentiation ensemble (1,024 x 256, ten pairs at c ~ 3.5e-4 A) against the oracle's
    FP64 analytic gradient with the same guard, directly (not through another adjoint)."""
    e, w = E.config3()
    g, _ = grad_tc(e.coords, w, eps)
    gref = oracle.crmsd_grad(e.coords, w.astype(np.float64), eps)
    compare(g, gref, f"config3 eps={eps} {mode}")


def test_clusters_match_independent_chunks():
    """The cluster path (rotations computed once, copied between CTAs) and the path where every
    chunk CTA recomputes them use the same arithmetic per pair: the gradients agree to the order
    of the float row-sum and near-duplicate additions."""
    e = E.decoy_ensemble(200, 700, 2, (0.3, 8.0), 77)
    w = E.weights(200 * 199 // 2, 78)
    os.environ.pop("CLUSCO_BACKWARD_CLUSTERS", None)
    g1, c = grad_tc(e.coords, w, 1e-6)
    os.environ["CLUSCO_BACKWARD_CLUSTERS"] = "0"
    try:
        g2, _ = grad_tc(e.coords, w, 1e-6, c)
    finally:
        os.environ.pop("CLUSCO_BACKWARD_CLUSTERS", None)
    d = np.linalg.norm((g1 - g2).reshape(200, -1), axis=1) / np.linalg.norm(g2.reshape(200, -1), axis=1)
    print(f"clusters vs independent chunks: max per-model rel diff {d.max():.2e}")
    assert d.max() <= 1e-6


def test_nonfinite_model_with_zero_weights():
    """A model with a NaN coordinate whose pairs all carry zero weight: every other gradient
    stays finite and equal to the oracle's on the finite models, the NaN model's is zero."""
    e = E.decoy_ensemble(90, 130, 1, (0.5, 6.0), 91)
    X = e.coords.copy()
    N = X.shape[0]
    bad = 37
    X[bad, 5, 1] = np.nan
    w = E.weights(N * (N - 1) // 2, 92)
    a, b = np.triu_indices(N, 1)
    w[(a == bad) | (b == bad)] = 0.0
    g, _ = grad_tc(X, w, 1e-6, status=6)  # CLUSCO_ENONFINITE: the forward saw the NaN
    keep = np.array([m for m in range(N) if m != bad])
    assert np.all(np.isfinite(g[keep]))
    assert np.all(g[bad] == 0.0)
    Xk = np.ascontiguousarray(X[keep])
    ak, bk = np.triu_indices(N - 1, 1)
    wk = w[(keep[ak] * N - keep[ak] * (keep[ak] + 1) // 2 + keep[bk] - keep[ak] - 1)]
    gref = oracle.crmsd_grad(Xk, wk.astype(np.float64), 1e-6)
    compare(g[keep], gref, "finite models beside a NaN model")


@pytest.mark.parametrize("N,L", [(8192, 500), (4000, 1000)])
def test_full_size_rows(N, L):
    """The large forward+backward workload (8,192 x 500, the bench's launch configuration) and a
    1,000-atom ensemble (three chunk CTAs): sampled rows against the oracle's FP64 gradient."""
    e = E.config4(N=N, L=L)
    w = E.weights(N * (N - 1) // 2, 505)
    X = torch.from_numpy(e.coords).cuda()
    c = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward(X, torch.from_numpy(w).cuda(), c, 1e-6, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    rows = np.unique(np.concatenate([[0, 1, 39, 40, N // 2, N - 1], np.random.default_rng(5).integers(0, N, 3)]))
    gref = oracle.crmsd_grad_rows(e.coords, w.astype(np.float64), rows, 1e-6)
    gg = g[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    compare(gg, gref, f"{N} x {L} sampled rows")


def test_autograd_recomputes_by_default():
    """The autograd Function keeps only the matrix and its backward is the recomputing adjoint."""
    e, w = E.config3()
    N = 300
    X = torch.from_numpy(e.coords[:N]).cuda().requires_grad_(True)
    wt = torch.from_numpy(w[: N * (N - 1) // 2]).cuda()
    loss = (wt * clusco.crmsd_matrix(X, clusco.FORM_BF16_EXACT2, 1e-6)).sum()
    loss.backward()
    c = clusco.crmsd_allpairs(X.detach(), clusco.FORM_BF16_EXACT2)
    g = clusco.crmsd_allpairs_backward(X.detach(), wt, c, 1e-6, clusco.FORM_BF16_EXACT2)
    torch.cuda.synchronize()
    d = (X.grad - g).reshape(N, -1).norm(dim=1) / g.reshape(N, -1).norm(dim=1)
    assert float(d.max()) <= 1e-6


@pytest.mark.parametrize("N,L", [(300, 128), (1000, 500)])
def test_fused_step_equals_the_two_calls(N, L):
    """clusco_crmsd_allpairs_step (the adjoint's pre-pass beside the forward) gives the matrix of
    clusco_crmsd_allpairs bit for bit and the gradient of clusco_crmsd_allpairs_backward, on the
    caller's stream and on another one, and from two streams at once on two ensembles."""
    e1 = E.decoy_ensemble(N, L, 2, (0.3, 8.0), 900 + L)
    e2 = E.decoy_ensemble(N, L, 3, (0.3, 8.0), 901 + L)
    w = torch.from_numpy(E.weights(N * (N - 1) // 2, 902)).cuda()
    refs = []
    for e in (e1, e2):
        X = torch.from_numpy(e.coords).cuda()
        c = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
        g = clusco.crmsd_allpairs_backward(X, w, c, 1e-6, clusco.FORM_BF16_EXACT2)
        refs.append((X, c, g))
    assert clusco.sync_status() == 0
    X, c, g = refs[0]
    out, gr = clusco.crmsd_allpairs_step(X, w, clusco.FORM_BF16_EXACT2, 1e-6)
    assert clusco.sync_status() == 0
    assert torch.equal(out, c)
    d = ((gr - g).reshape(N, -1).norm(dim=1) / g.reshape(N, -1).norm(dim=1)).max().item()
    assert d <= 1e-6
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for (Xk, _, _), st in zip(refs, (s1, s2)):
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            outs.append(clusco.crmsd_allpairs_step(Xk, w, clusco.FORM_BF16_EXACT2, 1e-6, stream=st))
    torch.cuda.synchronize()
    assert clusco.sync_status() == 0
    for (Xk, ck, gk), (o, gg) in zip(refs, outs):
        assert torch.equal(o, ck)
        d = ((gg - gk).reshape(N, -1).norm(dim=1) / gk.reshape(N, -1).norm(dim=1)).max().item()
        assert d <= 1e-6


def test_fused_step_in_a_cuda_graph():
    """The fused step captured into a CUDA graph from a torch stream (the side stream's fork and
    join become graph edges) and replayed twice gives the uncaptured call's matrix and gradient
    bit for bit. The ensemble has no near-duplicate pair, whose FP64 terms are added with float
    atomics in any order."""
    N, L = 400, 500
    e = E.decoy_ensemble(N, L, 2, (1.0, 8.0), 4242)
    X = torch.from_numpy(e.coords).cuda()
    w = torch.from_numpy(E.weights(N * (N - 1) // 2, 4243)).cuda()
    ws = torch.empty(clusco.workspace_bytes(clusco.OP_STEP, N, L), dtype=torch.uint8, device="cuda")
    out0, g0 = clusco.crmsd_allpairs_step(X, w, clusco.FORM_BF16_EXACT2, 1e-6, workspace=ws)
    assert clusco.sync_status() == 0
    assert float(out0.min()) >= 0.5  # no pair takes the near-duplicate path
    out, g = torch.empty_like(out0), torch.empty_like(g0)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        clusco.crmsd_allpairs_step(X, w, clusco.FORM_BF16_EXACT2, 1e-6, out=out, grad_coords=g, workspace=ws,
                                   stream=st)
    for _ in range(2):
        out.zero_()
        g.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, out0)
        assert torch.equal(g, g0)
    assert clusco.sync_status() == 0


def test_fused_step_argument_errors():
    X = torch.zeros((4, 8, 3), device="cuda")
    w = torch.ones(6, device="cuda")
    with pytest.raises(clusco.ClusCoError):  # the plain form has no fused step
        clusco.crmsd_allpairs_step(X, w, clusco.FORM_FP32_SIMT, 1e-6)
    with pytest.raises(clusco.ClusCoError):  # eps must be positive
        clusco.crmsd_allpairs_step(X, w, clusco.FORM_BF16_EXACT2, 0.0)
    Xl = torch.zeros((4, 1100, 3), device="cuda")
    with pytest.raises(clusco.ClusCoError):  # above the 1,024 atoms of the tensor-core adjoint
        clusco.crmsd_allpairs_step(Xl, w, clusco.FORM_BF16_EXACT2, 1e-6)

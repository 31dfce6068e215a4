"""Failure paths on the GPU, reached without a fault or a hang, through the test-hook library
(libclusco_debug.so: the production sources built with -DCLUSCO_DEBUG_HOOKS and 0.2 s device
waits; include/clusco_debug.h).

* A bounded wait that gives up: the tensor-core forward's TMA producer in CTA 0 skips its first
  pipeline stage (no arrive, no copy). The MMA issuer and the producer give up after 0.2 s, the
  CTA drains its copies in flight and leaves, the other CTAs finish, and the call's device status
  is CLUSCO_ETIMEOUT. Only the pairs of CTA 0's first tile (40 x 20 models) may be wrong, and the
  context stays usable: the production library then computes the same ensemble correctly.
* A near-duplicate queue that overflows: the adjoint with a queue of 4 entries, on an ensemble whose
  pairs are nearly all near-duplicates, reports the overflow (CLUSCO_ECUDA, "bounds") instead of
  dropping pairs silently; with the default capacity the same call is clean and matches the
  production library.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

pytestmark = pytest.mark.gpu

ETIMEOUT, ECUDA = 4, 3


@pytest.fixture(scope="module")
def dlib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    clusco.load()
    path = build.build_debug()
    lib = ctypes.CDLL(path)
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    lib.clusco_debug_hooks.argtypes = [ctypes.c_int, i64]
    lib.clusco_debug_flag_list_cap.argtypes = [ctypes.c_int]
    lib.clusco_crmsd_allpairs_below.argtypes = [vp, i64, i64, ctypes.c_float, vp, vp, i64, vp, ctypes.c_int, vp,
                                                sz, vp]
    lib.clusco_crmsd_allpairs.argtypes = [vp, i64, i64, vp, ctypes.c_int, vp, sz, vp]
    lib.clusco_crmsd_allpairs_backward.argtypes = [vp, i64, i64, vp, vp, vp, ctypes.c_float, ctypes.c_int, vp, sz,
                                                   vp]
    lib.clusco_sync_status.argtypes = [vp]
    lib.clusco_last_error.restype = ctypes.c_char_p
    yield lib
    lib.clusco_debug_hooks(0, 0)
    lib.clusco_debug_flag_list_cap(0)


def test_skipped_arrive_times_out_and_the_context_survives(dlib):
    e = E.decoy_ensemble(200, 64, 1, (0.5, 6.0), 4242)
    N, L = e.N, e.L
    P = N * (N - 1) // 2
    X = torch.from_numpy(e.coords).cuda()
    out = torch.full((P,), -1.0, device="cuda")
    assert dlib.clusco_debug_hooks(1, 0) == 0
    t0 = time.perf_counter()
    rc = dlib.clusco_crmsd_allpairs(X.data_ptr(), N, L, out.data_ptr(), clusco.FORM_BF16_EXACT2, None, 0, None)
    assert rc == 0, dlib.clusco_last_error()
    st = dlib.clusco_sync_status(None)
    elapsed = time.perf_counter() - t0
    assert dlib.clusco_debug_hooks(0, 0) == 0
    print(f"\nskipped arrive: status {st} ({dlib.clusco_last_error().decode()}) after {elapsed:.2f} s")
    assert st == ETIMEOUT
    assert elapsed < 10.0
    ref = oracle.crmsd_allpairs(e.coords)
    got = out.cpu().numpy().astype(np.float64)
    bad = ~(np.abs(got - ref) <= 1e-3)
    print(f"pairs off the oracle: {int(bad.sum())} of {P} (CTA 0's first tile holds at most 800)")
    assert bad.sum() <= 40 * 20
    # the same process and device: the production library is unaffected
    good = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2).cpu().numpy().astype(np.float64)
    assert clusco.sync_status() == 0
    assert np.abs(good - ref).max() <= 1e-3
    # and the debug library itself, hooks off, is clean again
    rc = dlib.clusco_crmsd_allpairs(X.data_ptr(), N, L, out.data_ptr(), clusco.FORM_BF16_EXACT2, None, 0, None)
    assert rc == 0 and dlib.clusco_sync_status(None) == 0
    assert np.abs(out.cpu().numpy() - good).max() == 0.0


def test_near_duplicate_queue_overflow_is_reported(dlib):
    e = E.decoy_ensemble(300, 120, 1, (0.05, 0.2), 777)  # nearly every pair below the 0.5 A threshold
    N, L = e.N, e.L
    X = torch.from_numpy(e.coords).cuda()
    w = torch.from_numpy(E.weights(N * (N - 1) // 2, 778)).cuda()
    c = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    want = clusco.crmsd_allpairs_backward(X, w, c, 1e-6, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    g = torch.empty_like(X)

    def run():
        rc = dlib.clusco_crmsd_allpairs_backward(X.data_ptr(), N, L, w.data_ptr(), c.data_ptr(), g.data_ptr(),
                                                 ctypes.c_float(1e-6), clusco.FORM_BF16_EXACT2, None, 0, None)
        assert rc == 0, dlib.clusco_last_error()
        return dlib.clusco_sync_status(None)

    assert dlib.clusco_debug_hooks(0, 4) == 0
    st = run()
    msg = dlib.clusco_last_error().decode()
    assert dlib.clusco_debug_hooks(0, 0) == 0
    print(f"\nnear-duplicate queue of 4: status {st} ({msg})")
    assert st == ECUDA and "bounds" in msg
    assert run() == 0
    rel = (torch.linalg.vector_norm((g - want).reshape(N, -1), dim=1)
           / torch.linalg.vector_norm(want.reshape(N, -1), dim=1).clamp_min(1e-30))
    assert float(rel.max()) <= 1e-5


def test_flagged_list_overflow_takes_the_mask_path(dlib):
    """The exact-digit forward lists its flagged pairs per epilogue warp; with the lists cut to one
    or three entries, the pairs past them go through the flag mask instead (the refinement's
    second path). The matrix, and the threshold list, are bit for bit the default library's."""
    e = E.decoy_ensemble(1200, 500, 10, (0.1, 12.0), 31337)  # the bench recipe: ~0.7 % flagged
    N, L = e.N, e.L
    P = N * (N - 1) // 2
    X = torch.from_numpy(e.coords).cuda()
    good = clusco.crmsd_allpairs(X, clusco.FORM_BF16_EXACT2)
    tau = 3.2
    gl, gv = clusco.crmsd_pairs_below(X, tau, clusco.FORM_BF16_EXACT2)
    assert clusco.sync_status() == 0
    gorder = torch.argsort(gl)
    for cap in (1, 3):
        assert dlib.clusco_debug_flag_list_cap(cap) == 0
        out = torch.full((P,), -1.0, device="cuda")
        rc = dlib.clusco_crmsd_allpairs(X.data_ptr(), N, L, out.data_ptr(), clusco.FORM_BF16_EXACT2, None, 0, None)
        assert rc == 0, dlib.clusco_last_error()
        assert dlib.clusco_sync_status(None) == 0
        assert torch.equal(out, good), cap
        cap_l = gl.numel() + 64
        lst = torch.empty(cap_l, dtype=torch.int64, device="cuda")
        vals = torch.empty(cap_l, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = dlib.clusco_crmsd_allpairs_below(X.data_ptr(), N, L, ctypes.c_float(tau), lst.data_ptr(),
                                              vals.data_ptr(), cap_l, cnt.data_ptr(), clusco.FORM_BF16_EXACT2, None,
                                              0, None)
        assert rc == 0, dlib.clusco_last_error()
        assert dlib.clusco_sync_status(None) == 0
        n = int(cnt.item())
        assert n == gl.numel()
        order = torch.argsort(lst[:n])
        assert torch.equal(lst[:n][order], gl[gorder]) and torch.equal(vals[:n][order], gv[gorder])
    assert dlib.clusco_debug_flag_list_cap(0) == 0

"""The allocation-free one-versus-reference entry point against the regular one.

clusco_crmsd_vs_ref_noalloc serves callers that cannot call cudaMalloc (device memory
owned by another allocator or pool, or latency-critical paths that cannot afford
cudaMalloc's possible synchronisation): it keeps its scratch in a fixed static device
array. Two calls in a row, on different ensembles and reference sizes, must each match
clusco_crmsd_vs_ref within the one-versus-reference tolerance (1e-4 A), so no state from
the first call leaks into the second. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1302_4000_b300 import build, clusco
from paper_1302_4000_b300 import ensembles as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    return clusco.load()


def test_noalloc_matches_regular_on_two_calls(lib):
    cases = [(E.config1(N=1500), 0), (E.decoy_ensemble(777, 150, 3, (0.1, 6.0), 4321), 2)]
    stream = torch.cuda.current_stream().cuda_stream
    for e, native in cases:
        X = torch.from_numpy(e.coords).cuda()
        ref = torch.from_numpy(e.natives[native].astype(np.float32)).cuda()
        want = clusco.crmsd_vs_ref(X, ref)
        got = torch.full((e.N,), float("nan"), device="cuda")
        rc = lib.clusco_crmsd_vs_ref_noalloc(X.data_ptr(), e.N, e.L, ref.data_ptr(), got.data_ptr(), stream)
        assert rc == 0, lib.clusco_last_error()
        assert clusco.sync_status() == 0
        err = (got - want).abs().max().item()
        assert np.isfinite(err) and err <= 1e-4, err


def test_noalloc_at_the_largest_reference_allocates_nothing(lib):
    """L = NOALLOC_MAX_L (N = 64): the whole static array in use. After a first call (which may
    load the module), a second call changes neither torch's allocator nor the device's free
    memory."""
    e = E.decoy_ensemble(64, clusco.NOALLOC_MAX_L, 2, (0.1, 6.0), 9090)
    X = torch.from_numpy(e.coords).cuda()
    ref = torch.from_numpy(e.natives[1].astype(np.float32)).cuda()
    want = clusco.crmsd_vs_ref(X, ref)
    got = torch.full((e.N,), float("nan"), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.clusco_crmsd_vs_ref_noalloc(X.data_ptr(), e.N, e.L, ref.data_ptr(), got.data_ptr(), stream) == 0
    assert clusco.sync_status() == 0
    got.fill_(float("nan"))
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    rc = lib.clusco_crmsd_vs_ref_noalloc(X.data_ptr(), e.N, e.L, ref.data_ptr(), got.data_ptr(), stream)
    assert rc == 0, lib.clusco_last_error()
    torch.cuda.synchronize()
    alloc1, free1 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    assert clusco.sync_status() == 0
    assert alloc1 == alloc0
    assert free1 == free0, (free0, free1)
    err = (got - want).abs().max().item()
    assert np.isfinite(err) and err <= 1e-4, err


def test_noalloc_rejects_oversized_reference(lib):
    fake = ctypes.c_void_p(0x1000)
    rc = lib.clusco_crmsd_vs_ref_noalloc(fake, 4, clusco.NOALLOC_MAX_L + 1, fake, fake, None)
    assert rc == 1
    assert b"maximum" in lib.clusco_last_error()

"""The C-ABI library builds, loads and exports every declared entry point (no GPU needed).

Argument validation runs on the host before any CUDA call, so those checks run here too.
"""
import ctypes
import os
import re

import pytest

from paper_1302_4000_b300 import build, clusco

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return clusco.load()


DEBUG_HEADER = "clusco_debug.h"  # the test-hook library's extra entry points


def declared_symbols(headers=None):
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h") and (h in headers if headers else h != DEBUG_HEADER):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(clusco_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "clusco_crmsd_allpairs" in syms and "clusco_crmsd_allpairs_backward" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert set(clusco.EXPORTS) <= set(syms)
    # the test hooks exist only in the debug library, which exports everything else too
    dbg = declared_symbols([DEBUG_HEADER])
    assert dbg == ["clusco_debug_flag_list_cap", "clusco_debug_hooks"]
    for s in dbg:
        assert not hasattr(lib, s), s
    if os.path.exists(build.DEBUG_LIB) and not build.stale(build.DEBUG_LIB):
        dlib = ctypes.CDLL(build.DEBUG_LIB)
        for s in syms + dbg:
            assert hasattr(dlib, s), s


def test_version_and_workspace(lib):
    assert clusco.version() >= 10000
    for form in clusco.FORMS.values():
        assert clusco.workspace_bytes(clusco.OP_ALLPAIRS, 5000, 300, form) > 0
        assert clusco.workspace_bytes(clusco.OP_ALLPAIRS, 1, 300, form) == 0
    assert clusco.workspace_bytes(clusco.OP_VS_REF, 5000, 300, 0) > 0
    assert clusco.workspace_bytes(clusco.OP_BACKWARD, 1024, 256, 0) > 0
    assert clusco.workspace_bytes(99, 10, 10, 0) == 0


def _call_allpairs(lib, ptr, N, L, out, form):
    return lib.clusco_crmsd_allpairs(ptr, N, L, out, form, None, 0, None)


def test_host_side_validation(lib):
    fake = ctypes.c_void_p(0x1000)
    assert _call_allpairs(lib, fake, 1, 10, fake, 0) == 1          # N < 2
    assert _call_allpairs(lib, fake, 10, 0, fake, 0) == 1          # L < 1
    assert _call_allpairs(lib, None, 10, 10, fake, 0) == 1         # null coords
    assert _call_allpairs(lib, ctypes.c_void_p(0x1001), 10, 10, fake, 0) == 1  # unaligned
    assert _call_allpairs(lib, fake, 10, 10, fake, 42) == 1        # unknown form
    assert b"form" in lib.clusco_last_error()
    assert _call_allpairs(lib, fake, 1 << 40, 10, fake, 0) == 5    # N overflow
    assert lib.clusco_crmsd_allpairs_panel(fake, 10, 10, 5, 3, fake, 0, None, 0, None) == 1  # bad range
    assert lib.clusco_crmsd_allpairs_panel(fake, 10, 10, 0, 10, fake, 0, None, 0, None) == 1  # row_end > N-1
    assert lib.clusco_crmsd_vs_ref(fake, 10, 10, None, fake, None, 0, None) == 1
    assert lib.clusco_crmsd_allpairs_backward(fake, 10, 10, fake, fake, fake, ctypes.c_float(0.0), 0,
                                              None, 0, None) == 1  # eps must be > 0
    # a workspace that is too small is refused before any launch
    assert lib.clusco_crmsd_allpairs(fake, 10, 10, fake, 0, fake, 16, None) == 2
    # threshold mode: NaN tau, negative capacity, missing or unaligned list / count
    nan = ctypes.c_float(float("nan"))
    assert lib.clusco_crmsd_allpairs_below(fake, 10, 10, nan, fake, fake, 4, fake, 0, None, 0, None) == 1
    assert lib.clusco_crmsd_allpairs_below(fake, 10, 10, ctypes.c_float(1.0), fake, fake, -1, fake, 0, None, 0,
                                           None) == 1
    assert lib.clusco_crmsd_allpairs_below(fake, 10, 10, ctypes.c_float(1.0), None, fake, 4, fake, 0, None, 0,
                                           None) == 1
    assert lib.clusco_crmsd_allpairs_below(fake, 10, 10, ctypes.c_float(1.0), ctypes.c_void_p(0x1004), fake, 4,
                                           fake, 0, None, 0, None) == 1
    assert lib.clusco_crmsd_allpairs_below(fake, 10, 10, ctypes.c_float(1.0), fake, fake, 4, None, 0, None, 0,
                                           None) == 1


def test_condensed_pairs_inverts_the_condensed_index():
    """The binding's host-side inverse of idx(a, b) = a N - a (a + 1) / 2 + (b - a - 1)."""
    import numpy as np
    import torch
    for N in (2, 3, 7, 50, 1001):
        a_ref, b_ref = np.triu_indices(N, 1)
        a, b = clusco.condensed_pairs(torch.arange(N * (N - 1) // 2), N)
        assert np.array_equal(a.numpy(), a_ref) and np.array_equal(b.numpy(), b_ref), N
    N = 3_000_000  # last and first pairs at a size where the float estimate needs its corrections
    P = N * (N - 1) // 2
    a, b = clusco.condensed_pairs(torch.tensor([0, 1, N - 2, N - 1, P - 2, P - 1]), N)
    assert a.tolist() == [0, 0, 0, 1, N - 3, N - 2] and b.tolist() == [1, 2, N - 1, 2, N - 1, N - 1]


def test_drmsd_host_side_validation(lib):
    fake = ctypes.c_void_p(0x1000)
    call = lib.clusco_drmsd_allpairs
    assert call(fake, 1, 10, fake, 0, None, 0, None) == 1        # N < 2
    assert call(fake, 10, 1, fake, 0, None, 0, None) == 1        # L < 2: no atom pair
    assert call(fake, 10, 5000, fake, 0, None, 0, None) == 1     # above the staged-coordinates limit
    assert call(fake, 10, 10, None, 0, None, 0, None) == 1       # null out
    assert call(fake, 10, 10, fake, clusco.FORM_TF32, None, 0, None) == 7  # form without a dRMSD kernel
    assert call(fake, 10, 10, fake, 0, fake, 16, None) == 2      # workspace too small
    for form in (clusco.FORM_FP32_SIMT, clusco.FORM_BF16_EXACT2):
        nb = clusco.workspace_bytes(clusco.OP_DRMSD, 5000, 300, form)
        # the distances of every model dominate: 4 bytes per model and atom pair, padded
        assert 5000 * 44850 * 4 <= nb <= 5120 * 44864 * 4 + (1 << 20)
    assert clusco.workspace_bytes(clusco.OP_DRMSD, 5000, 300, clusco.FORM_TF32) == 0
    assert clusco.workspace_bytes(clusco.OP_DRMSD, 10, 1, 0) == 0


def test_cmo_host_side_validation(lib):
    fake = ctypes.c_void_p(0x1000)
    call = lib.clusco_cmo_allpairs
    c8 = ctypes.c_float(8.0)
    assert call(fake, 1, 10, c8, fake, 0, None, 0, None) == 1                      # N < 2
    assert call(fake, 10, 1, c8, fake, 0, None, 0, None) == 1                      # L < 2
    assert call(fake, 10, 5000, c8, fake, 0, None, 0, None) == 1                   # L above 4096
    assert call(fake, 10, 10, ctypes.c_float(0.0), fake, 0, None, 0, None) == 1    # cutoff must be > 0
    assert call(fake, 10, 10, ctypes.c_float(float("inf")), fake, 0, None, 0, None) == 1
    assert call(fake, 10, 10, c8, None, 0, None, 0, None) == 1                     # null out
    assert call(fake, 10, 10, c8, fake, clusco.FORM_BF16_EXACT2, None, 0, None) == 7  # no such CMO form
    assert call(fake, 10, 10, c8, fake, 0, fake, 16, None) == 2                    # workspace too small
    for form in (clusco.FORM_FP32_SIMT, clusco.FORM_FP8_EXACT):
        nb = clusco.workspace_bytes(clusco.OP_CMO, 5000, 300, form)
        assert 5000 * 44850 <= nb <= 5120 * 45056 * 1.2 + (1 << 20)
    assert clusco.workspace_bytes(clusco.OP_CMO, 5000, 300, clusco.FORM_TF32) == 0
    # the cRMSD entry points do not take the contact-map form
    assert lib.clusco_crmsd_allpairs(fake, 10, 10, fake, clusco.FORM_FP8_EXACT, None, 0, None) == 1


def test_gdt_tm_host_side_validation(lib):
    fake = ctypes.c_void_p(0x1000)
    call = lib.clusco_gdt_tm_vs_ref
    assert call(fake, 0, 10, fake, fake, None) == 1        # N < 1
    assert call(fake, 10, 2, fake, fake, None) == 1        # L < 3
    assert call(fake, 10, 1025, fake, fake, None) == 1     # L above 1024
    assert call(fake, 10, 10, None, fake, None) == 1       # null reference
    assert call(fake, 10, 10, fake, None, None) == 1       # null out


def test_step_rot_host_side_validation(lib):
    """The fused step's workspace is the two calls' workspaces, the forward's rounded up to 256
    bytes; its argument errors return before anything is enqueued."""
    r256 = lambda x: (x + 255) // 256 * 256
    for N, L, form in ((5000, 300, clusco.FORM_BF16_EXACT2), (129, 255, clusco.FORM_TF32),
                       (2, 1, clusco.FORM_BF16X3)):
        fwd = clusco.workspace_bytes(clusco.OP_ALLPAIRS_ROT, N, L, form)
        bwd = clusco.workspace_bytes(clusco.OP_BACKWARD_ROT, N, L, form)
        assert fwd > 0 and bwd > 0
        assert clusco.workspace_bytes(clusco.OP_STEP_ROT, N, L, form) == r256(fwd) + bwd
    assert clusco.workspace_bytes(clusco.OP_STEP_ROT, 5000, 300, clusco.FORM_FP32_SIMT) == 0  # no rotations
    assert clusco.workspace_bytes(clusco.OP_STEP_ROT, 100, 600, clusco.FORM_BF16_EXACT2) == 0  # L > 512
    assert clusco.workspace_bytes(clusco.OP_STEP_ROT, 1, 300, clusco.FORM_BF16_EXACT2) == 0
    fake, eps = ctypes.c_void_p(0x1000), ctypes.c_float(1e-6)
    step = lib.clusco_crmsd_allpairs_step_rot
    ex = clusco.FORM_BF16_EXACT2
    assert step(fake, 10, 10, None, fake, fake, fake, ex, eps, None, 0, None) == 1  # null weights
    assert step(fake, 10, 10, fake, fake, ctypes.c_void_p(0x1004), fake, ex, eps, None, 0, None) == 1  # rot 16 B
    assert step(fake, 10, 10, fake, fake, fake, fake, 42, eps, None, 0, None) == 1  # unknown form
    assert step(fake, 10, 10, fake, fake, fake, fake, ex, ctypes.c_float(0.0), None, 0, None) == 1  # eps
    assert step(fake, 1, 10, fake, fake, fake, fake, ex, eps, None, 0, None) == 1  # N < 2
    assert step(fake, 10, 10, fake, fake, fake, fake, clusco.FORM_FP32_SIMT, eps, None, 0, None) == 7
    assert step(fake, 10, 10, fake, fake, fake, fake, clusco.FORM_INT_SIMT, eps, None, 0, None) == 7
    assert step(fake, 10, 600, fake, fake, fake, fake, ex, eps, None, 0, None) == 7  # L > 512


def test_exact_integer_form_host_side(lib):
    """The exact-integer CUDA-core form serves the all-pairs calls only: no rotations, no fused
    step, no dRMSD / contact map overlap; L is capped where its int64 sums could overflow."""
    ix = clusco.FORM_INT_SIMT
    assert clusco.workspace_bytes(clusco.OP_ALLPAIRS, 5000, 300, ix) > 0
    for op in (clusco.OP_ALLPAIRS_ROT, clusco.OP_STEP, clusco.OP_STEP_ROT, clusco.OP_DRMSD, clusco.OP_CMO):
        assert clusco.workspace_bytes(op, 5000, 300, ix) == 0, op
    fake, eps = ctypes.c_void_p(0x1000), ctypes.c_float(1e-6)
    assert lib.clusco_crmsd_allpairs_rot(fake, 10, 10, fake, fake, ix, None, 0, None) == 7
    assert lib.clusco_crmsd_allpairs_step(fake, 10, 10, fake, fake, fake, ix, eps, None, 0, None) == 7
    assert lib.clusco_drmsd_allpairs(fake, 10, 10, fake, ix, None, 0, None) == 7
    assert lib.clusco_crmsd_allpairs(fake, 10, (1 << 17) + 1, fake, ix, None, 0, None) == 7

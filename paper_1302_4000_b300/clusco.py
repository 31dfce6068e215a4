"""Thin Python binding of libclusco (argument marshalling only).

Every function here has the name of its C entry point without the ``clusco_``
prefix and does nothing but check shapes, allocate outputs with torch, pass raw
device pointers and the current CUDA stream to the library, and raise on a
non-OK status. All arithmetic runs in the library's CUDA kernels; there is no
CPU fallback: if ``libclusco.so`` is missing or no CUDA device is present, the
calls raise.

The operations are ClusCo's cRMSD (section "Algorithms", eq. 1 / eq. 2), dRMSD (eq. 5)
and contact map overlap (eq. 6 / eq. 7) over the N(N-1)/2 pairs of an ensemble (section
"Background"), and GDT_TS / TM-score / MaxSub (eq. 3 / eq. 4) against a reference.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libclusco.so")

FORM_FP32_SIMT = 0
FORM_TF32 = 1
FORM_BF16X3 = 2
FORM_BF16_EXACT2 = 3
FORM_FP8_EXACT = 4  # the contact map overlap's tensor-core form
FORM_INT_SIMT = 5  # exact-integer CUDA-core form (all-pairs cRMSD only)
FORMS = {"fp32_simt": FORM_FP32_SIMT, "tf32": FORM_TF32, "bf16x3": FORM_BF16X3, "bf16_exact2": FORM_BF16_EXACT2,
         "int_simt": FORM_INT_SIMT}

OP_ALLPAIRS = 0
OP_VS_REF = 1
OP_BACKWARD = 2
OP_BACKWARD_ROT = 3
OP_ALLPAIRS_ROT = 4
OP_DRMSD = 5
OP_CMO = 6
OP_STEP_ROT = 7
OP_STEP = 8

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EOVERFLOW",
          6: "ENONFINITE", 7: "EUNSUPPORTED"}

EXPORTS = ("clusco_version", "clusco_workspace_bytes", "clusco_crmsd_allpairs", "clusco_crmsd_allpairs_panel",
           "clusco_crmsd_allpairs_below",
           "clusco_crmsd_vs_ref", "clusco_crmsd_vs_ref_noalloc", "clusco_crmsd_allpairs_backward",
           "clusco_sync_status", "clusco_last_error", "clusco_profile_enable", "clusco_profile_read",
           "clusco_crmsd_allpairs_rot", "clusco_crmsd_allpairs_backward_rot", "clusco_drmsd_allpairs",
           "clusco_cmo_allpairs", "clusco_gdt_tm_vs_ref", "clusco_crmsd_allpairs_step_rot",
           "clusco_crmsd_allpairs_step")
KERNEL_PAIRS = 0
KERNEL_ADJOINT = 1
KERNEL_DRMSD = 2
KERNEL_CMO = 3
NOALLOC_MAX_L = 16384

_lib = None
_lock = threading.Lock()


class ClusCoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"clusco {STATUS.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libclusco.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ClusCoError(3, f"{path} not built; run paper_1302_4000_b300.build.build()")
            lib = ctypes.CDLL(path)
            vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
            lib.clusco_version.restype = ctypes.c_int
            lib.clusco_last_error.restype = ctypes.c_char_p
            lib.clusco_workspace_bytes.restype = sz
            lib.clusco_workspace_bytes.argtypes = [ctypes.c_int, i64, i64, ctypes.c_int]
            lib.clusco_crmsd_allpairs.argtypes = [vp, i64, i64, vp, ctypes.c_int, vp, sz, vp]
            lib.clusco_crmsd_allpairs_panel.argtypes = [vp, i64, i64, i64, i64, vp, ctypes.c_int, vp, sz, vp]
            lib.clusco_crmsd_allpairs_below.argtypes = [vp, i64, i64, ctypes.c_float, vp, vp, i64, vp,
                                                        ctypes.c_int, vp, sz, vp]
            lib.clusco_crmsd_vs_ref.argtypes = [vp, i64, i64, vp, vp, vp, sz, vp]
            lib.clusco_crmsd_vs_ref_noalloc.argtypes = [vp, i64, i64, vp, vp, vp]
            lib.clusco_crmsd_allpairs_backward.argtypes = [vp, i64, i64, vp, vp, vp, ctypes.c_float, ctypes.c_int,
                                                           vp, sz, vp]
            lib.clusco_sync_status.argtypes = [vp]
            lib.clusco_crmsd_allpairs_rot.argtypes = [vp, i64, i64, vp, vp, ctypes.c_int, vp, sz, vp]
            lib.clusco_crmsd_allpairs_backward_rot.argtypes = [vp, i64, i64, vp, vp, vp, vp, ctypes.c_float, vp, sz,
                                                               vp]
            lib.clusco_crmsd_allpairs_step_rot.argtypes = [vp, i64, i64, vp, vp, vp, vp, ctypes.c_int, ctypes.c_float,
                                                           vp, sz, vp]
            lib.clusco_crmsd_allpairs_step.argtypes = [vp, i64, i64, vp, vp, vp, ctypes.c_int, ctypes.c_float, vp,
                                                       sz, vp]
            lib.clusco_drmsd_allpairs.argtypes = [vp, i64, i64, vp, ctypes.c_int, vp, sz, vp]
            lib.clusco_cmo_allpairs.argtypes = [vp, i64, i64, ctypes.c_float, vp, ctypes.c_int, vp, sz, vp]
            lib.clusco_gdt_tm_vs_ref.argtypes = [vp, i64, i64, vp, vp, vp]
            lib.clusco_profile_enable.argtypes = [ctypes.c_int]
            lib.clusco_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_longlong)]
            for f in ("clusco_crmsd_allpairs", "clusco_crmsd_allpairs_panel", "clusco_crmsd_vs_ref",
                      "clusco_crmsd_vs_ref_noalloc", "clusco_crmsd_allpairs_backward", "clusco_sync_status",
                      "clusco_profile_enable", "clusco_profile_read", "clusco_crmsd_allpairs_rot",
                      "clusco_crmsd_allpairs_backward_rot", "clusco_crmsd_allpairs_below", "clusco_drmsd_allpairs",
                      "clusco_cmo_allpairs", "clusco_gdt_tm_vs_ref", "clusco_crmsd_allpairs_step_rot",
                      "clusco_crmsd_allpairs_step"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        raise ClusCoError(rc, load().clusco_last_error().decode())


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _coords(coords: torch.Tensor):
    if not coords.is_cuda:
        raise ValueError("coords must be a CUDA tensor (use *_host for host buffers)")
    if coords.dtype != torch.float32 or coords.dim() != 3 or coords.shape[2] != 3:
        raise ValueError("coords must be float32 [N, L, 3]")
    return coords.contiguous()


def version() -> int:
    return load().clusco_version()


def profile_enable(on: bool = True) -> None:
    """Start (True) or stop (False) bracketing the tensor-core kernels' launches with events."""
    _check(load().clusco_profile_enable(1 if on else 0))


def profile_read(kernel: int):
    """(total ms, launches) of the given kernel's bracketed launches since profile_enable(True)."""
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(load().clusco_profile_read(kernel, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def workspace_bytes(op: int, N: int, L: int, form: int = FORM_BF16_EXACT2) -> int:
    return int(load().clusco_workspace_bytes(op, N, L, form))


def _ws(workspace, op, N, L, form, device):
    if workspace is not None:
        return workspace, workspace.numel() * workspace.element_size()
    nb = workspace_bytes(op, N, L, form)
    return torch.empty(max(nb, 1), dtype=torch.uint8, device=device), nb


def crmsd_allpairs(coords: torch.Tensor, form: int = FORM_BF16_EXACT2, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Condensed all-versus-all cRMSD (float32, length N(N-1)/2) on coords' device."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=coords.device)
    assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= P and out.is_contiguous()
    ws, nb = _ws(workspace, OP_ALLPAIRS, N, L, form, coords.device)
    _check(load().clusco_crmsd_allpairs(coords.data_ptr(), N, L, out.data_ptr(), form, ws.data_ptr(), nb,
                                        _stream(stream)))
    return out


def drmsd_allpairs(coords: torch.Tensor, form: int = FORM_BF16_EXACT2, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Condensed all-versus-all dRMSD (eq. 5; float32, length N(N-1)/2) on coords' device.
    Forms: FORM_BF16_EXACT2 (tensor cores, exact Gram of 16-bit rounded distances) and
    FORM_FP32_SIMT (plain: FP32 distances differenced directly)."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=coords.device)
    assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= P and out.is_contiguous()
    ws, nb = _ws(workspace, OP_DRMSD, N, L, form, coords.device)
    _check(load().clusco_drmsd_allpairs(coords.data_ptr(), N, L, out.data_ptr(), form, ws.data_ptr(), nb,
                                        _stream(stream)))
    return out


def cmo_allpairs(coords: torch.Tensor, cutoff: float = 8.0, form: int = FORM_FP8_EXACT,
                 out: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Condensed all-versus-all contact map overlap (eq. 7, percent; float32, length N(N-1)/2) with
    contacts |x_i - x_j| < cutoff (A) over atom pairs i < j. Forms: FORM_FP8_EXACT (tensor cores)
    and FORM_FP32_SIMT (plain: bit-packed maps, population count); both count exactly."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=coords.device)
    assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= P and out.is_contiguous()
    ws, nb = _ws(workspace, OP_CMO, N, L, form, coords.device)
    _check(load().clusco_cmo_allpairs(coords.data_ptr(), N, L, float(cutoff), out.data_ptr(), form, ws.data_ptr(),
                                      nb, _stream(stream)))
    return out


def gdt_tm_vs_ref(coords: torch.Tensor, ref: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """[N, 3] float32: GDT_TS (fraction), TM-score and MaxSub of every model against the reference
    (eq. 3, eq. 4), each the maximum over the paper's superposition search."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    ref = ref.contiguous()
    assert ref.is_cuda and ref.dtype == torch.float32 and tuple(ref.shape) == (L, 3)
    if out is None:
        out = torch.empty((N, 3), dtype=torch.float32, device=coords.device)
    assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= 3 * N and out.is_contiguous()
    _check(load().clusco_gdt_tm_vs_ref(coords.data_ptr(), N, L, ref.data_ptr(), out.data_ptr(), _stream(stream)))
    return out


def crmsd_pairs_below(coords: torch.Tensor, tau: float, form: int = FORM_BF16_EXACT2, capacity: int | None = None,
                      workspace: torch.Tensor | None = None, stream=None):
    """(idx, vals): every pair a < b with cRMSD < tau, as int64 condensed indices and their
    float32 cRMSD (exactly the values crmsd_allpairs gives in the same form), in no particular
    order. capacity is the first guess at their number; when more qualify, the call runs again
    with room for all of them (the library reports the full count)."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    cap = max(1024, P // 64) if capacity is None else int(capacity)
    cap = min(cap, P)
    ws, nb = _ws(workspace, OP_ALLPAIRS, N, L, form, coords.device)
    count = torch.zeros(1, dtype=torch.int64, device=coords.device)
    while True:
        idx = torch.empty(max(cap, 1), dtype=torch.int64, device=coords.device)
        vals = torch.empty(max(cap, 1), dtype=torch.float32, device=coords.device)
        _check(load().clusco_crmsd_allpairs_below(coords.data_ptr(), N, L, float(tau), idx.data_ptr(), vals.data_ptr(),
                                                  cap, count.data_ptr(), form, ws.data_ptr(), nb, _stream(stream)))
        n = int(count.item())
        if n <= cap:
            return idx[:n], vals[:n]
        cap = n


def condensed_pairs(idx: torch.Tensor, N: int):
    """(a, b) with a < b for condensed indices idx = a N - a (a + 1) / 2 + (b - a - 1)."""
    i = idx.to(torch.float64)
    t = 2.0 * N - 1.0
    a = torch.floor(0.5 * (t - torch.sqrt(torch.clamp(t * t - 8.0 * i, min=0.0)))).to(torch.int64).clamp(0, N - 2)
    start = lambda r: r * N - r * (r + 1) // 2
    a = torch.where(start(a) > idx, a - 1, a)
    a = torch.where(start(a + 1) <= idx, a + 1, a)
    b = idx - start(a) + a + 1
    return a, b


ROT_STRIDE = 12


def rotations_view(rot: torch.Tensor) -> torch.Tensor:
    """The [P, 3, 3] rotations inside a stored-rotation buffer of [P, ROT_STRIDE] records."""
    return rot[:, :9].reshape(-1, 3, 3)


def crmsd_allpairs_rot(coords: torch.Tensor, form: int = FORM_BF16_EXACT2, out: torch.Tensor | None = None,
                       rot: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    """(matrix, rotation records): the condensed cRMSD and each pair's R_ab as float32
    [P, ROT_STRIDE] records (R row-major in the first nine; rotations_view gives [P, 3, 3])."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=coords.device)
    if rot is None:
        rot = torch.empty((P, ROT_STRIDE), dtype=torch.float32, device=coords.device)
    assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= P and out.is_contiguous()
    assert rot.is_cuda and rot.dtype == torch.float32 and rot.numel() >= ROT_STRIDE * P and rot.is_contiguous()
    ws, nb = _ws(workspace, OP_ALLPAIRS_ROT, N, L, form, coords.device)
    _check(load().clusco_crmsd_allpairs_rot(coords.data_ptr(), N, L, out.data_ptr(), rot.data_ptr(), form,
                                            ws.data_ptr(), nb, _stream(stream)))
    return out, rot


def crmsd_allpairs_panel(coords: torch.Tensor, row_begin: int, row_end: int, form: int = FORM_BF16_EXACT2,
                         out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """Rows [row_begin, row_end) of the condensed matrix (all b > a), in condensed order."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]

    def start(a):
        return a * N - a * (a + 1) // 2

    n = start(row_end) - start(row_begin)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=coords.device)
    ws, nb = _ws(workspace, OP_ALLPAIRS, N, L, form, coords.device)
    _check(load().clusco_crmsd_allpairs_panel(coords.data_ptr(), N, L, row_begin, row_end, out.data_ptr(), form,
                                              ws.data_ptr(), nb, _stream(stream)))
    return out


def crmsd_vs_ref(coords: torch.Tensor, ref: torch.Tensor, out: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """cRMSD of every model against ref ([L, 3] float32, same device)."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    ref = ref.contiguous()
    assert ref.is_cuda and ref.dtype == torch.float32 and tuple(ref.shape) == (L, 3)
    if out is None:
        out = torch.empty(N, dtype=torch.float32, device=coords.device)
    ws, nb = _ws(workspace, OP_VS_REF, N, L, 0, coords.device)
    _check(load().clusco_crmsd_vs_ref(coords.data_ptr(), N, L, ref.data_ptr(), out.data_ptr(), ws.data_ptr(), nb,
                                      _stream(stream)))
    return out


def crmsd_vs_ref_noalloc(coords: torch.Tensor, ref: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """One-versus-reference through the entry point that allocates no device memory.

    For callers that cannot allocate (device memory owned by another pool, or no room for
    cudaMalloc's synchronisation on a latency-critical path): the caller passes the output,
    the library uses a fixed static device array (references up to NOALLOC_MAX_L atoms).
    """
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    assert ref.is_cuda and ref.is_contiguous() and tuple(ref.shape) == (L, 3)
    assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= N
    _check(load().clusco_crmsd_vs_ref_noalloc(coords.data_ptr(), N, L, ref.data_ptr(), out.data_ptr(),
                                              _stream(stream)))
    return out


def crmsd_allpairs_backward(coords: torch.Tensor, grad_out: torch.Tensor, crmsd: torch.Tensor, eps: float = 1e-6,
                            form: int = FORM_BF16_EXACT2, grad_coords: torch.Tensor | None = None,
                            workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """d Loss / d coords for dLoss/dcRMSD = grad_out (condensed), reusing the forward's crmsd."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    grad_out = grad_out.contiguous().to(torch.float32)
    crmsd = crmsd.contiguous()
    assert grad_out.numel() == P and crmsd.numel() == P and grad_out.is_cuda and crmsd.is_cuda
    if grad_coords is None:
        grad_coords = torch.empty_like(coords)
    ws, nb = _ws(workspace, OP_BACKWARD, N, L, form, coords.device)
    _check(load().clusco_crmsd_allpairs_backward(coords.data_ptr(), N, L, grad_out.data_ptr(), crmsd.data_ptr(),
                                                 grad_coords.data_ptr(), float(eps), form, ws.data_ptr(), nb,
                                                 _stream(stream)))
    return grad_coords


def crmsd_allpairs_backward_rot(coords: torch.Tensor, grad_out: torch.Tensor, crmsd: torch.Tensor,
                                rot: torch.Tensor, eps: float = 1e-6, grad_coords: torch.Tensor | None = None,
                                workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The adjoint from the rotations crmsd_allpairs_rot stored (no covariance recomputation)."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    grad_out = grad_out.contiguous().to(torch.float32)
    crmsd = crmsd.contiguous()
    rot = rot.contiguous()
    assert grad_out.numel() == P and crmsd.numel() == P and rot.numel() == ROT_STRIDE * P
    assert grad_out.is_cuda and crmsd.is_cuda and rot.is_cuda
    if grad_coords is None:
        grad_coords = torch.empty_like(coords)
    ws, nb = _ws(workspace, OP_BACKWARD_ROT, N, L, FORM_BF16_EXACT2, coords.device)
    _check(load().clusco_crmsd_allpairs_backward_rot(coords.data_ptr(), N, L, grad_out.data_ptr(), crmsd.data_ptr(),
                                                     rot.data_ptr(), grad_coords.data_ptr(), float(eps),
                                                     ws.data_ptr(), nb, _stream(stream)))
    return grad_coords


def crmsd_allpairs_step_rot(coords: torch.Tensor, grad_out: torch.Tensor, form: int = FORM_BF16_EXACT2,
                            eps: float = 1e-6, out: torch.Tensor | None = None, rot: torch.Tensor | None = None,
                            grad_coords: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                            stream=None):
    """One training step in one call: the matrix and the rotations (crmsd_allpairs_rot), then the
    adjoint of the weights grad_out from them (crmsd_allpairs_backward_rot), with the adjoint's
    pre-pass beside the forward. Returns (out, rot, grad_coords)."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    grad_out = grad_out.contiguous().to(torch.float32)
    assert grad_out.numel() == P and grad_out.is_cuda
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=coords.device)
    if rot is None:
        rot = torch.empty((P, ROT_STRIDE), dtype=torch.float32, device=coords.device)
    if grad_coords is None:
        grad_coords = torch.empty_like(coords)
    assert out.is_contiguous() and rot.is_contiguous() and grad_coords.is_contiguous()
    assert out.numel() == P and rot.numel() == ROT_STRIDE * P and grad_coords.shape == coords.shape
    ws, nb = _ws(workspace, OP_STEP_ROT, N, L, form, coords.device)
    _check(load().clusco_crmsd_allpairs_step_rot(coords.data_ptr(), N, L, grad_out.data_ptr(), out.data_ptr(),
                                                 rot.data_ptr(), grad_coords.data_ptr(), int(form), float(eps),
                                                 ws.data_ptr(), nb, _stream(stream)))
    return out, rot, grad_coords


def crmsd_allpairs_step(coords: torch.Tensor, grad_out: torch.Tensor, form: int = FORM_BF16_EXACT2,
                        eps: float = 1e-6, out: torch.Tensor | None = None, grad_coords: torch.Tensor | None = None,
                        workspace: torch.Tensor | None = None, stream=None):
    """One training step in one call, nothing stored between its halves: the matrix
    (crmsd_allpairs), then the adjoint of the weights grad_out with every rotation recomputed
    (crmsd_allpairs_backward), with the adjoint's pre-pass beside the forward. Returns
    (out, grad_coords)."""
    coords = _coords(coords)
    N, L = coords.shape[0], coords.shape[1]
    P = N * (N - 1) // 2
    grad_out = grad_out.contiguous().to(torch.float32)
    assert grad_out.numel() == P and grad_out.is_cuda
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=coords.device)
    if grad_coords is None:
        grad_coords = torch.empty_like(coords)
    assert out.is_contiguous() and grad_coords.is_contiguous()
    assert out.numel() == P and grad_coords.shape == coords.shape
    ws, nb = _ws(workspace, OP_STEP, N, L, form, coords.device)
    _check(load().clusco_crmsd_allpairs_step(coords.data_ptr(), N, L, grad_out.data_ptr(), out.data_ptr(),
                                             grad_coords.data_ptr(), int(form), float(eps), ws.data_ptr(), nb,
                                             _stream(stream)))
    return out, grad_coords


def sync_status(stream=None) -> int:
    """Synchronise the stream and return the device status word (0 = clean); clears it."""
    rc = load().clusco_sync_status(_stream(stream))
    return rc


class CRMSDAllPairs(torch.autograd.Function):
    """Condensed all-pairs cRMSD with the library's hand-written adjoint.

    By default nothing but the matrix is kept for the backward, which recomputes every pair's
    rotation. With store_rotations (a tensor-core form and L <= 512) the forward also stores each
    pair's rotation (48 bytes per pair) and the backward contracts from it instead."""

    @staticmethod
    def forward(ctx, coords, form: int, eps: float, store_rotations: bool = False):
        store = (store_rotations and ctx.needs_input_grad[0] and form != FORM_FP32_SIMT
                 and coords.shape[1] <= 512)
        if store:
            out, rot = crmsd_allpairs_rot(coords, form)
            ctx.save_for_backward(coords, out, rot)
        else:
            out = crmsd_allpairs(coords, form)
            ctx.save_for_backward(coords, out)
        ctx.form, ctx.eps, ctx.store = form, eps, store
        return out

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.store:
            coords, out, rot = ctx.saved_tensors
            g = crmsd_allpairs_backward_rot(coords, grad_out, out, rot, ctx.eps)
        else:
            coords, out = ctx.saved_tensors
            g = crmsd_allpairs_backward(coords, grad_out, out, ctx.eps, ctx.form)
        return g, None, None, None


def crmsd_matrix(coords: torch.Tensor, form: int = FORM_BF16_EXACT2, eps: float = 1e-6,
                 store_rotations: bool = False) -> torch.Tensor:
    """Differentiable condensed cRMSD matrix (the backward recomputes the rotations unless
    store_rotations)."""
    return CRMSDAllPairs.apply(coords, form, eps, store_rotations)


def crmsd_allpairs_host(coords_host: torch.Tensor, form: int = FORM_BF16_EXACT2, out_host: torch.Tensor | None = None,
                        device="cuda", stream=None) -> torch.Tensor:
    """End-to-end call with host buffers: H2D of coords, the all-pairs kernels, D2H of the matrix."""
    assert not coords_host.is_cuda
    d = coords_host.to(device, non_blocking=True)
    out = crmsd_allpairs(d, form, stream=stream)
    if out_host is None:
        out_host = torch.empty(out.numel(), dtype=torch.float32, pin_memory=True)
    out_host.copy_(out, non_blocking=True)
    return out_host

"""FP64 CPU oracle for all-versus-all cRMSD, dRMSD and CMO (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package. It shares no code with the CUDA path:
the C sources ``crmsd_oracle.c``, ``drmsd_oracle.c`` and ``cmo_oracle.c`` are compiled
on their own with gcc (OpenMP for timing only, no floating-point contraction) and loaded
through ctypes.

The cRMSD functions follow ClusCo's definition (section "Algorithms",
eq. 1: RMS deviation of matched atoms after the optimal superposition, with the
cited Kabsch method). ``crmsd_eq2_pair`` restates the paper's closed form
(eq. 2: radii of gyration, eigenvalues of M^T M from a cubic, sign of det M)
and serves as a pin and as a second CPU method; the oracle's answers never
come from it.

``gdt_tm_vs_ref`` scores models against a reference with GDT_TS, TM-score and MaxSub (eq. 3,
eq. 4) as maxima over the paper's superposition search (fragment seeds of 4, L/4, L/2 and L
atoms, refinement on the atoms within 3.5 A), each superposition from the Kabsch path above.

The dRMSD functions follow eq. 5 (the RMS difference of the two models'
intra-model distance matrices over the L(L-1)/2 atom pairs), formed directly
from the distances. The CMO functions follow eq. 6 and eq. 7 (contact maps over the
atom pairs i < j, the Sorensen index of two maps); the contact test is taken in FP32,
the precision of the CUDA kernels, and the score in FP64.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariances, brute-force rotation search, eq. 2, finite
differences); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crmsd_oracle.c")
_DSRC = os.path.join(_HERE, "drmsd_oracle.c")
_CSRC = os.path.join(_HERE, "cmo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(src=(_SRC, _DSRC, _CSRC), out: str = _LIB, extra_flags=()) -> str:
    """Compile the oracle source(s) with gcc (-O2, FP64, OpenMP). Returns the .so path."""
    srcs = [src] if isinstance(src, str) else list(src)
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", *extra_flags, *srcs, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def load(path: str | None = None):
    """Load (building first if missing or stale) and return the ctypes library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
                    os.path.getmtime(f) for f in (_SRC, _DSRC, _CSRC)):
                build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    """Declare the signatures of whichever entry points the library holds (a test may load a
    library built from one of the two sources)."""
    i64 = ctypes.c_int64
    if hasattr(lib, "oracle_drmsd_pair"):
        lib.oracle_drmsd_pair.argtypes = [_f32p, _f32p, i64, ctypes.POINTER(ctypes.c_double)]
        lib.oracle_drmsd_allpairs.argtypes = [_f32p, i64, i64, _f64p, ctypes.c_int]
        lib.oracle_drmsd_pairs.argtypes = [_f32p, i64, i64, _i64p, _i64p, i64, _f64p, ctypes.c_int]
        for f in ("oracle_drmsd_pair", "oracle_drmsd_allpairs", "oracle_drmsd_pairs"):
            getattr(lib, f).restype = ctypes.c_int
    if hasattr(lib, "oracle_cmo_pair"):
        f32 = ctypes.c_float
        lib.oracle_cmo_counts.argtypes = [_f32p, _f32p, i64, f32] + [ctypes.POINTER(ctypes.c_int64)] * 3
        lib.oracle_cmo_pair.argtypes = [_f32p, _f32p, i64, f32, ctypes.POINTER(ctypes.c_double)]
        lib.oracle_cmo_allpairs.argtypes = [_f32p, i64, i64, f32, _f64p, ctypes.c_int]
        lib.oracle_cmo_pairs.argtypes = [_f32p, i64, i64, f32, _i64p, _i64p, i64, _f64p, ctypes.c_int]
        for f in ("oracle_cmo_counts", "oracle_cmo_pair", "oracle_cmo_allpairs", "oracle_cmo_pairs"):
            getattr(lib, f).restype = ctypes.c_int
    if not hasattr(lib, "oracle_crmsd_pair"):
        return lib
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_crmsd_pair.argtypes = [_f32p, _f32p, i64, ctypes.POINTER(ctypes.c_double), _f64p]
    lib.oracle_crmsd_allpairs.argtypes = [_f32p, i64, i64, _f64p, ctypes.c_int]
    lib.oracle_crmsd_pairs.argtypes = [_f32p, i64, i64, _i64p, _i64p, i64, _f64p, ctypes.c_int]
    lib.oracle_crmsd_vs_ref.argtypes = [_f32p, i64, i64, _f32p, _f64p, ctypes.c_int]
    lib.oracle_crmsd_grad.argtypes = [_f32p, i64, i64, _f64p, ctypes.c_double, _f64p, ctypes.c_int]
    lib.oracle_crmsd_eq2.argtypes = [_f32p, _f32p, i64, ctypes.POINTER(ctypes.c_double)]
    lib.oracle_crmsd_grad_rows.argtypes = [_f32p, i64, i64, _f64p, ctypes.c_double, _i64p, i64, _f64p, ctypes.c_int]
    lib.oracle_gdt_tm_vs_ref.argtypes = [_f32p, i64, i64, _f32p, _f64p, ctypes.c_int]
    lib.oracle_gdt_tm_vs_ref_rule.argtypes = [_f32p, i64, i64, _f32p, _f64p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int]
    for f in ("oracle_crmsd_pair", "oracle_crmsd_allpairs", "oracle_crmsd_pairs",
              "oracle_crmsd_vs_ref", "oracle_crmsd_grad", "oracle_crmsd_eq2", "oracle_crmsd_grad_rows",
              "oracle_gdt_tm_vs_ref", "oracle_gdt_tm_vs_ref_rule"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def max_threads() -> int:
    return int(load().oracle_max_threads())


def crmsd_pair(A, B, lib=None):
    """(cRMSD, R) for one pair; R (3x3) maps centred B onto centred A."""
    lib = lib or load()
    A, B = _f32(A), _f32(B)
    assert A.shape == B.shape and A.ndim == 2 and A.shape[1] == 3
    c = ctypes.c_double()
    R = np.zeros(9, dtype=np.float64)
    _check(lib.oracle_crmsd_pair(A, B, A.shape[0], ctypes.byref(c), R), "pair")
    return c.value, R.reshape(3, 3)


def crmsd_allpairs(X, nthreads: int = 0, lib=None) -> np.ndarray:
    """Condensed N(N-1)/2 FP64 matrix, row-major upper triangle (a < b)."""
    lib = lib or load()
    X = _f32(X)
    N, L = X.shape[0], X.shape[1]
    out = np.empty(N * (N - 1) // 2, dtype=np.float64)
    _check(lib.oracle_crmsd_allpairs(X, N, L, out, nthreads), "allpairs")
    return out


def crmsd_pairs(X, ia, ib, nthreads: int = 0, lib=None) -> np.ndarray:
    """cRMSD for the listed pairs (ia[k], ib[k])."""
    lib = lib or load()
    X = _f32(X)
    ia = np.ascontiguousarray(ia, dtype=np.int64)
    ib = np.ascontiguousarray(ib, dtype=np.int64)
    out = np.empty(ia.shape[0], dtype=np.float64)
    _check(lib.oracle_crmsd_pairs(X, X.shape[0], X.shape[1], ia, ib, ia.shape[0], out, nthreads), "pairs")
    return out


def crmsd_vs_ref(X, ref, nthreads: int = 0, lib=None) -> np.ndarray:
    """out[a] = cRMSD(model a, ref) in FP64."""
    lib = lib or load()
    X, ref = _f32(X), _f32(ref)
    out = np.empty(X.shape[0], dtype=np.float64)
    _check(lib.oracle_crmsd_vs_ref(X, X.shape[0], X.shape[1], ref, out, nthreads), "vs_ref")
    return out


def crmsd_grad(X, w, eps: float = 1e-6, nthreads: int = 0, lib=None) -> np.ndarray:
    """d/dX of sum_{a<b} w_ab cRMSD_ab, shape [N, L, 3] (FP64)."""
    lib = lib or load()
    X = _f32(X)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N, L = X.shape[0], X.shape[1]
    assert w.shape[0] == N * (N - 1) // 2
    g = np.empty((N, L, 3), dtype=np.float64)
    _check(lib.oracle_crmsd_grad(X, N, L, w, float(eps), g.reshape(-1), nthreads), "grad")
    return g


def crmsd_grad_rows(X, w, rows, eps: float = 1e-6, nthreads: int = 0, lib=None) -> np.ndarray:
    """Rows of d/dX sum_{a<b} w_ab cRMSD_ab for the listed models, shape [len(rows), L, 3]."""
    lib = lib or load()
    X = _f32(X)
    w = np.ascontiguousarray(w, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    N, L = X.shape[0], X.shape[1]
    g = np.empty((rows.shape[0], L, 3), dtype=np.float64)
    _check(lib.oracle_crmsd_grad_rows(X, N, L, w, float(eps), rows, rows.shape[0], g.reshape(-1), nthreads),
           "grad_rows")
    return g


def crmsd_eq2_pair(A, B, lib=None) -> float:
    """The paper's closed form (eq. 2) in FP64 for one pair."""
    lib = lib or load()
    A, B = _f32(A), _f32(B)
    c = ctypes.c_double()
    _check(lib.oracle_crmsd_eq2(A, B, A.shape[0], ctypes.byref(c)), "eq2")
    return c.value


def drmsd_pair(A, B, lib=None) -> float:
    """dRMSD (eq. 5) of one pair of models [L, 3], L >= 2, in FP64."""
    lib = lib or load()
    A, B = _f32(A), _f32(B)
    assert A.shape == B.shape and A.ndim == 2 and A.shape[1] == 3
    c = ctypes.c_double()
    _check(lib.oracle_drmsd_pair(A, B, A.shape[0], ctypes.byref(c)), "drmsd_pair")
    return c.value


def drmsd_allpairs(X, nthreads: int = 0, lib=None) -> np.ndarray:
    """Condensed N(N-1)/2 FP64 dRMSD matrix, row-major upper triangle (a < b)."""
    lib = lib or load()
    X = _f32(X)
    N, L = X.shape[0], X.shape[1]
    out = np.empty(N * (N - 1) // 2, dtype=np.float64)
    _check(lib.oracle_drmsd_allpairs(X, N, L, out, nthreads), "drmsd_allpairs")
    return out


def drmsd_pairs(X, ia, ib, nthreads: int = 0, lib=None) -> np.ndarray:
    """dRMSD for the listed pairs (ia[k], ib[k])."""
    lib = lib or load()
    X = _f32(X)
    ia = np.ascontiguousarray(ia, dtype=np.int64)
    ib = np.ascontiguousarray(ib, dtype=np.int64)
    out = np.empty(ia.shape[0], dtype=np.float64)
    _check(lib.oracle_drmsd_pairs(X, X.shape[0], X.shape[1], ia, ib, ia.shape[0], out, nthreads),
           "drmsd_pairs")
    return out


def cmo_counts(A, B, cutoff: float, lib=None):
    """(n(A), n(B), n(A and B)): contact counts over atom pairs i < j (eq. 6)."""
    lib = lib or load()
    A, B = _f32(A), _f32(B)
    na, nb, nab = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.oracle_cmo_counts(A, B, A.shape[0], float(cutoff), ctypes.byref(na), ctypes.byref(nb),
                                 ctypes.byref(nab)), "cmo_counts")
    return na.value, nb.value, nab.value


def cmo_pair(A, B, cutoff: float, lib=None) -> float:
    """CMO score (eq. 7, in percent) of one pair of models."""
    lib = lib or load()
    A, B = _f32(A), _f32(B)
    c = ctypes.c_double()
    _check(lib.oracle_cmo_pair(A, B, A.shape[0], float(cutoff), ctypes.byref(c)), "cmo_pair")
    return c.value


def cmo_allpairs(X, cutoff: float, nthreads: int = 0, lib=None) -> np.ndarray:
    """Condensed N(N-1)/2 FP64 CMO matrix, row-major upper triangle (a < b)."""
    lib = lib or load()
    X = _f32(X)
    N, L = X.shape[0], X.shape[1]
    out = np.empty(N * (N - 1) // 2, dtype=np.float64)
    _check(lib.oracle_cmo_allpairs(X, N, L, float(cutoff), out, nthreads), "cmo_allpairs")
    return out


def cmo_pairs(X, ia, ib, cutoff: float, nthreads: int = 0, lib=None) -> np.ndarray:
    """CMO for the listed pairs (ia[k], ib[k])."""
    lib = lib or load()
    X = _f32(X)
    ia = np.ascontiguousarray(ia, dtype=np.int64)
    ib = np.ascontiguousarray(ib, dtype=np.int64)
    out = np.empty(ia.shape[0], dtype=np.float64)
    _check(lib.oracle_cmo_pairs(X, X.shape[0], X.shape[1], float(cutoff), ia, ib, ia.shape[0], out, nthreads),
           "cmo_pairs")
    return out


def gdt_tm_vs_ref(X, ref, nthreads: int = 0, lib=None) -> np.ndarray:
    """[N, 3] FP64: GDT_TS (fraction), TM-score, MaxSub of every model against the reference, each
    the maximum over the paper's superposition search (fragment seeds, 3.5 A refinement)."""
    lib = lib or load()
    X, ref = _f32(X), _f32(ref)
    N, L = X.shape[0], X.shape[1]
    out = np.empty((N, 3), dtype=np.float64)
    _check(lib.oracle_gdt_tm_vs_ref(X, N, L, ref, out.reshape(-1), nthreads), "gdt_tm_vs_ref")
    return out


def gdt_tm_vs_ref_rule(X, ref, stable: int, max_refine: int, nthreads: int = 0, lib=None) -> np.ndarray:
    """gdt_tm_vs_ref with the search's stop rule given: stop after `stable` refinements in a row
    that select as many atoms as the superposition before them, or after `max_refine`
    refinements. gdt_tm_vs_ref is (4, 20); (1, 4) is the shorter reading."""
    lib = lib or load()
    X, ref = _f32(X), _f32(ref)
    N, L = X.shape[0], X.shape[1]
    out = np.empty((N, 3), dtype=np.float64)
    _check(lib.oracle_gdt_tm_vs_ref_rule(X, N, L, ref, out.reshape(-1), nthreads, stable, max_refine),
           "gdt_tm_vs_ref_rule")
    return out

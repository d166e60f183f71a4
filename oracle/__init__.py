"""CPU oracle for the discrete Frechet distance -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
under ``paper_2404_05708_gb300`` and its binding) never imports it and
shares no code with it.

Contents:
  * ``dfd_oracle.c`` -- plain C, float64 / int64: Alg. 1 (memoised), Alg. 3
    (full matrix), Alg. 5 (linear row), a decision-search cross-check, the
    discrete Hausdorff distance, a float32 selection mirror, the appendix's
    DTW and Levenshtein recurrences, and a threaded pair-list driver.
  * ``brute.py``     -- brute-force minimum over all monotone couplings.
  * ``fast_form.py`` -- Alg. 2 written as a fold of scans (numpy, float64).

All distance functions return SQUARED distances (delta^2): the recurrence of
Eq. 1 only selects among its inputs, so it commutes with the square root.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfd_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-pthread"]


def build(out_path: str | None = None, mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc; ``mutant`` plants a known mistake (tests only)."""
    out_path = out_path or _LIB_PATH
    if not force and mutant == 0 and os.path.exists(out_path) and \
            os.path.getmtime(out_path) >= os.path.getmtime(_SRC):
        return out_path
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, f"-DDFO_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_F32P = ctypes.POINTER(ctypes.c_float)
_F64P = ctypes.POINTER(ctypes.c_double)


def _declare(lib):
    c_i64, c_int = ctypes.c_int64, ctypes.c_int
    for name in ("dfo_linear_f64", "dfo_full_f64", "dfo_memo_f64", "dfo_decide_f64", "dfo_hausdorff_f64",
                 "dfo_dtw_f64"):
        f = getattr(lib, name)
        f.restype = ctypes.c_double
        f.argtypes = [_F32P, c_i64, _F32P, c_i64, c_int]
    for name in ("dfo_linear_i64", "dfo_full_i64", "dfo_memo_i64", "dfo_decide_i64", "dfo_hausdorff_i64"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int64
        f.argtypes = [_I32P, c_i64, _I32P, c_i64, c_int]
    lib.dfo_linear_f32mirror.restype = ctypes.c_float
    lib.dfo_linear_f32mirror.argtypes = [_F32P, c_i64, _F32P, c_i64, c_int]
    lib.dfo_batch_f64.restype = c_int
    lib.dfo_batch_f64.argtypes = [_F32P, _I64P, _I32P, c_i64, c_int, _F64P, c_int]
    lib.dfo_batch_i64.restype = c_int
    lib.dfo_batch_i64.argtypes = [_I32P, _I64P, _I32P, c_i64, c_int, _I64P, c_int]
    lib.dfo_batch_f32mirror.restype = c_int
    lib.dfo_batch_f32mirror.argtypes = [_F32P, _I64P, _I32P, c_i64, c_int, _F32P, c_int]
    lib.dfo_perturb_f32.restype = None
    lib.dfo_perturb_f32.argtypes = [_F32P, _F32P, ctypes.c_float, c_i64, _F32P]
    lib.dfo_dtw_f32mirror.restype = ctypes.c_float
    lib.dfo_dtw_f32mirror.argtypes = [_F32P, c_i64, _F32P, c_i64, c_int]
    lib.dfo_levenshtein.restype = ctypes.c_int64
    lib.dfo_levenshtein.argtypes = [_I32P, c_i64, _I32P, c_i64]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` selects a variant."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctype)


def _prep(p, q):
    p = np.asarray(p)
    q = np.asarray(q)
    if p.ndim == 1:
        p = p[:, None]
    if q.ndim == 1:
        q = q[:, None]
    if p.shape[1] != q.shape[1]:
        raise ValueError("dimension mismatch")
    if p.shape[0] < 1 or q.shape[0] < 1:
        raise ValueError("curves must have at least one point")
    if p.dtype.kind in "iu" and q.dtype.kind in "iu":
        return np.ascontiguousarray(p, np.int32), np.ascontiguousarray(q, np.int32), True
    return np.ascontiguousarray(p, np.float32), np.ascontiguousarray(q, np.float32), False


def _call(kind: str, p, q, lib=None):
    lib = lib or load()
    p, q, is_int = _prep(p, q)
    n, m, dim = p.shape[0], q.shape[0], p.shape[1]
    if is_int:
        f = getattr(lib, f"dfo_{kind}_i64")
        return int(f(_ptr(p, _I32P), n, _ptr(q, _I32P), m, dim))
    f = getattr(lib, f"dfo_{kind}_f64")
    return float(f(_ptr(p, _F32P), n, _ptr(q, _F32P), m, dim))


def dfd2_linear(p, q, lib=None):
    """delta^2 by Alg. 5 (linear row).  float32 in -> float, int32 in -> int."""
    return _call("linear", p, q, lib)


def dfd2_full(p, q, lib=None):
    """delta^2 by Alg. 3 (full matrix with the four branches)."""
    return _call("full", p, q, lib)


def dfd2_memo(p, q, lib=None):
    """delta^2 by Alg. 1 (memoised top-down recursion, explicit stack)."""
    return _call("memo", p, q, lib)


def dfd2_decide(p, q, lib=None):
    """delta^2 by binary search over thresholds + BFS reachability."""
    return _call("decide", p, q, lib)


def hausdorff2(p, q, lib=None):
    """Squared symmetric discrete Hausdorff distance."""
    return _call("hausdorff", p, q, lib)


def dfd2_f32mirror(p, q, lib=None):
    """Alg. 5 in float32 with the kernel's squared-distance evaluation order."""
    lib = lib or load()
    p, q, is_int = _prep(p, q)
    if is_int:
        raise TypeError("the float32 mirror takes float32 curves")
    return np.float32(lib.dfo_linear_f32mirror(_ptr(p, _F32P), p.shape[0], _ptr(q, _F32P), q.shape[0],
                                               p.shape[1]))


def dtw(p, q, lib=None):
    """DTW with squared-Euclidean ground cost (float64)."""
    lib = lib or load()
    p, q, _ = _prep(np.asarray(p, np.float32), np.asarray(q, np.float32))
    return float(lib.dfo_dtw_f64(_ptr(p, _F32P), p.shape[0], _ptr(q, _F32P), q.shape[0], p.shape[1]))


def dtw_f32mirror(p, q, lib=None):
    """DTW in float32, one rounding per cell (the GPU kernel's order)."""
    lib = lib or load()
    p, q, _ = _prep(np.asarray(p, np.float32), np.asarray(q, np.float32))
    return float(lib.dfo_dtw_f32mirror(_ptr(p, _F32P), p.shape[0], _ptr(q, _F32P), q.shape[0], p.shape[1]))


def perturb(x, z, sigma, lib=None):
    """x + sigma * z per coordinate, one float32 rounding (uncertain-curve samples)."""
    lib = lib or load()
    x = np.ascontiguousarray(x, np.float32)
    z = np.ascontiguousarray(z, np.float32)
    if x.shape != z.shape:
        raise ValueError("x and z must have one shape")
    out = np.empty_like(x)
    lib.dfo_perturb_f32(_ptr(x, _F32P), _ptr(z, _F32P), float(sigma), x.size, _ptr(out, _F32P))
    return out


def levenshtein(a, b, lib=None):
    """Textbook edit distance of two int32 symbol sequences."""
    lib = lib or load()
    a = np.ascontiguousarray(a, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    return int(lib.dfo_levenshtein(_ptr(a, _I32P), a.shape[0], _ptr(b, _I32P), b.shape[0]))


def batch(points, offsets, pairs, nthreads: int | None = None, mirror: bool = False, lib=None):
    """Alg. 5 over a list of (a, b) curve pairs on ``nthreads`` CPU threads.

    Returns (delta^2 array, threads used): float64 for float32 curves
    (float32 when ``mirror``), int64 for int32 curves.
    """
    lib = lib or load()
    points = np.asarray(points)
    offsets = np.ascontiguousarray(offsets, np.int64)
    pairs = np.ascontiguousarray(pairs, np.int32).reshape(-1, 2)
    n_pairs = pairs.shape[0]
    dim = points.shape[1]
    nthreads = nthreads or os.cpu_count() or 1
    if points.dtype.kind in "iu":
        pts = np.ascontiguousarray(points, np.int32)
        out = np.empty(n_pairs, np.int64)
        used = lib.dfo_batch_i64(_ptr(pts, _I32P), _ptr(offsets, _I64P), _ptr(pairs, _I32P), n_pairs, dim,
                                 _ptr(out, _I64P), nthreads)
    elif mirror:
        pts = np.ascontiguousarray(points, np.float32)
        out = np.empty(n_pairs, np.float32)
        used = lib.dfo_batch_f32mirror(_ptr(pts, _F32P), _ptr(offsets, _I64P), _ptr(pairs, _I32P), n_pairs,
                                       dim, _ptr(out, _F32P), nthreads)
    else:
        pts = np.ascontiguousarray(points, np.float32)
        out = np.empty(n_pairs, np.float64)
        used = lib.dfo_batch_f64(_ptr(pts, _F32P), _ptr(offsets, _I64P), _ptr(pairs, _I32P), n_pairs, dim,
                                 _ptr(out, _F64P), nthreads)
    return out, int(used)

"""Oracle for the Stream-K GEMM library.  TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline and
reference legs may import this package.  The product (``paper_2301_03598_gb300``)
never imports it, and it imports nothing from the product.

Contents:

* ``gemm`` / ``gemm_entries`` -- plain FP64 GEMM, C = alpha*A*B + beta*C
  (paper, Section 2), in C (``oracle_gemm.c``), loaded through ctypes.
* ``schedule`` -- the decompositions of Algorithms 2, 4, 5, the hybrids of
  Section 5.2 and the grid-size model of Appendix A.1, in Python.
* ``rounding`` -- round-to-nearest-even onto FP32 / FP16 / BF16 and their ulp.
* ``e4m3`` -- the E4M3 code values and the block-scaled E4M3 GEMM (operands
  dequantized exactly, then the FP64 GEMM above).

The C library is compiled with gcc on first use (or by ``build()``), next to
its source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import e4m3, rounding, schedule  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_gemm.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle_gemm.c into _build/liboracle.so (gcc, OpenMP, -O2).
    No fast-math: the summation order of the source is kept."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                        "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, pd = ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
            pi64 = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_gemm_f64.restype = ctypes.c_int
            lib.oracle_gemm_f64.argtypes = [i64, i64, i64, dbl, pd, i64, i64, pd, i64, i64,
                                            dbl, pd, i64, i64, pd, pd, ctypes.c_int]
            lib.oracle_gemm_entries_f64.restype = ctypes.c_int
            lib.oracle_gemm_entries_f64.argtypes = [i64, pi64, pi64, i64, dbl, pd, i64, i64,
                                                    pd, i64, i64, dbl, pd, i64, i64, pd, pd,
                                                    ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _f64(x):
    a = np.asarray(x)
    if a.dtype != np.float64:
        raise TypeError("oracle inputs must already be float64 (widened exactly)")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _strides(a):
    return tuple(s // a.itemsize for s in a.strides)


def max_threads(nthreads: int = 0) -> int:
    return _load().oracle_max_threads(nthreads)


def gemm(A, B, alpha: float = 1.0, beta: float = 0.0, C_in=None, nthreads: int = 0):
    """Return (C64, absAB): C64 = alpha*A@B + beta*C_in and absAB = |A|@|B|,
    both m x n float64.  A (m x k), B (k x n) and C_in are float64 arrays of any
    strides holding the exact input values."""
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if beta != 0.0:
        C_in = _f64(C_in)
        if C_in.shape != (m, n):
            raise ValueError("C_in shape")
        crs, ccs = _strides(C_in)
    else:
        C_in, crs, ccs = None, 0, 0
    C64 = np.empty((m, n), np.float64)
    absAB = np.empty((m, n), np.float64)
    ars, acs = _strides(A)
    brs, bcs = _strides(B)
    rc = _load().oracle_gemm_f64(m, n, k, alpha, _ptr(A), ars, acs, _ptr(B), brs, bcs,
                                 beta, _ptr(C_in), crs, ccs, _ptr(C64), _ptr(absAB), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_gemm_f64 failed ({rc})")
    return C64, absAB


def gemm_entries(rows, cols, A, B, alpha: float = 1.0, beta: float = 0.0, C_in=None,
                 nthreads: int = 0):
    """Entries (rows[e], cols[e]) of alpha*A@B + beta*C_in, and of |A|@|B|."""
    A, B = _f64(A), _f64(B)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    if rows.shape != cols.shape or rows.ndim != 1:
        raise ValueError("rows/cols must be equal-length vectors")
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if rows.size and (rows.min() < 0 or rows.max() >= m or cols.min() < 0 or cols.max() >= n):
        raise IndexError("entry index out of range")
    if beta != 0.0:
        C_in = _f64(C_in)
        crs, ccs = _strides(C_in)
    else:
        C_in, crs, ccs = None, 0, 0
    out = np.empty(rows.size, np.float64)
    absout = np.empty(rows.size, np.float64)
    ars, acs = _strides(A)
    brs, bcs = _strides(B)
    pi64 = ctypes.POINTER(ctypes.c_int64)
    rc = _load().oracle_gemm_entries_f64(
        rows.size, rows.ctypes.data_as(pi64), cols.ctypes.data_as(pi64), k, alpha,
        _ptr(A), ars, acs, _ptr(B), brs, bcs, beta, _ptr(C_in), crs, ccs,
        _ptr(out), _ptr(absout), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_gemm_entries_f64 failed ({rc})")
    return out, absout

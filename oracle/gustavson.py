"""C = A*B on the CPU: plain serial Gustavson with an ordered-map accumulator.

Test infrastructure.  Follows Sec. 2.2 of the paper (Gustavson's row-wise
algorithm, Fig. 1): rows of A in order, a_ik in ascending k, b_kj of row k of
B, acc[j] += a_ik*b_kj, row of C = accumulator in column order; the structure
is the symbolic one (entries that cancel to zero are kept).  The arithmetic is
in ``spgemm_oracle.cpp``; this module compiles it with g++ and calls it.

Pinned in tests/test_oracle_gustavson.py against a dense triple loop, the
closed-form 13-point stencil of the squared 5-point Laplacian, the closed-form
125-point structure of the squared 27-point stencil, and permutation
invariance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

DT_F32, DT_F64, DT_I64 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared object (g++, -O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-std=c++17", _SRC, "-o", tmp])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_spgemm.restype = ctypes.c_void_p
        lib.oracle_spgemm.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 7 + [ctypes.c_int] * 3
        lib.oracle_result_nnz.restype = ctypes.c_int64
        lib.oracle_result_nnz.argtypes = [ctypes.c_void_p]
        lib.oracle_result_copy.argtypes = [ctypes.c_void_p] * 5
        lib.oracle_result_free.argtypes = [ctypes.c_void_p]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def dtype_code(val: np.ndarray) -> int:
    if val.dtype == np.float32:
        return DT_F32
    if val.dtype == np.float64:
        return DT_F64
    if val.dtype == np.int64:
        return DT_I64
    raise TypeError(val.dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def spgemm(A, B, rows=None, want_mag: bool = True, nthreads: int = 1):
    """Rows ``rows`` (default: all) of A*B.

    A and B are any objects with ``row_ptr`` (int64), ``col`` (int32), ``val`` and
    ``nrows``/``ncols``.  Returns (row_ptr, col, val, mag): val is float64 for FP32
    and FP64 inputs, int64 for int64 inputs; mag = (|A||B|)_ij (float64) or None.
    """
    lib = _load()
    arp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    acol = np.ascontiguousarray(A.col, dtype=np.int32)
    aval = np.ascontiguousarray(A.val)
    brp = np.ascontiguousarray(B.row_ptr, dtype=np.int64)
    bcol = np.ascontiguousarray(B.col, dtype=np.int32)
    bval = np.ascontiguousarray(B.val)
    dt = dtype_code(aval)
    assert dtype_code(bval) == dt, "A and B must share a value type"
    if rows is None:
        nsel, rows_arr = A.nrows, None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nsel = rows_arr.size
    h = lib.oracle_spgemm(nsel, _p(rows_arr), _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol),
                          _p(bval), dt, 1 if want_mag else 0, int(nthreads))
    try:
        nnz = lib.oracle_result_nnz(h)
        rp = np.zeros(nsel + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz, dtype=np.int64 if dt == DT_I64 else np.float64)
        mag = np.zeros(nnz, dtype=np.float64) if want_mag else None
        lib.oracle_result_copy(h, _p(rp), _p(col), _p(val), _p(mag))
    finally:
        lib.oracle_result_free(h)
    return rp, col, val, mag


def max_threads() -> int:
    return int(_load().oracle_max_threads())

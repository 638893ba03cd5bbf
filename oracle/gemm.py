"""FP64-accumulating reference GEMM (test infrastructure only).

Python face of ``gemm_ref.c``: the plain definition
C_ref = alpha * op(A) @ op(B) + beta * C_in, every product and sum in FP64,
computed from the FP32 inputs.  See the C file for the layout conventions.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_gemm_f64.restype = ctypes.c_int
        lib.oracle_gemm_f64.argtypes = [
            ctypes.c_char, ctypes.c_char, ctypes.c_long, ctypes.c_long, ctypes.c_long,
            ctypes.c_double, ctypes.c_void_p, ctypes.c_long,
            ctypes.c_void_p, ctypes.c_long, ctypes.c_double,
            ctypes.c_void_p, ctypes.c_long,
            ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_long,
        ]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def _f32(x):
    a = np.asarray(x)
    if a.dtype != np.float32:
        raise TypeError("oracle inputs must be float32 (the GPU sees FP32 bits)")
    return np.ascontiguousarray(a)


def gemm(A, B, transA: str = "N", transB: str = "N", alpha: float = 1.0,
         beta: float = 0.0, C=None, M=None, N=None, K=None, rows=None) -> np.ndarray:
    """FP64 result of alpha*op(A)*op(B) + beta*C for FP32 row-major inputs.

    A and B are 2-D row-major arrays whose leading dimension is their column
    count; M, N, K default to the logical extents implied by the transposes
    (a caller may pass smaller ones to use a sub-block of padded storage).
    ``rows`` restricts the output to those rows of C (in the given order).
    ``alpha`` and ``beta`` are taken as the FP32 values the kernel receives.
    """
    A = _f32(A)
    B = _f32(B)
    lda, ldb = A.shape[1], B.shape[1]
    M = (A.shape[0] if transA == "N" else A.shape[1]) if M is None else M
    K = (A.shape[1] if transA == "N" else A.shape[0]) if K is None else K
    N = (B.shape[1] if transB == "N" else B.shape[0]) if N is None else N
    alpha = float(np.float32(alpha))
    beta = float(np.float32(beta))
    if beta != 0.0:
        C = _f32(C)
        ldc, cptr = C.shape[1], C.ctypes.data
    else:
        ldc, cptr = max(N, 1), None
    if rows is None:
        rows_arr, nrows, count = None, 0, M
    else:
        rows_arr = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        if rows_arr.size and (rows_arr.min() < 0 or rows_arr.max() >= M):
            raise ValueError("row index out of range")
        nrows, count = rows_arr.size, rows_arr.size
    out = np.zeros((count, N), dtype=np.float64)
    rc = _load().oracle_gemm_f64(
        transA.encode(), transB.encode(), M, N, K, alpha,
        A.ctypes.data, lda, B.ctypes.data, ldb, beta, cptr, ldc,
        out.ctypes.data, max(N, 1),
        None if rows_arr is None else rows_arr.ctypes.data, nrows)
    if rc != 0:
        raise RuntimeError("oracle_gemm_f64 failed (%d)" % rc)
    return out

"""ctypes front of ``omp.c``: the job kinds' CPU reference results with
OpenMP over the host cores, used for the CPU baseline (test
infrastructure only). The GEMM's product is a library matrix multiply
(numpy, BLAS threads) of the operands generated here."""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_omp())
        P, U64 = ctypes.c_void_p, ctypes.c_uint64
        lib.omp_threads.restype = ctypes.c_int
        lib.omp_triad.argtypes = [U64, U64, ctypes.c_float, P]
        lib.omp_spmv.argtypes = [U64, U64, P, P, P, P]
        lib.omp_spmv.restype = ctypes.c_int64
        lib.omp_gemm_operand.argtypes = [U64, U64, U64, U64, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """OpenMP threads the kernels run on."""
    return int(_load().omp_threads())


def triad(key: int, n: int, s: float = 3.0) -> np.ndarray:
    a = np.empty(n, dtype=np.float32)
    _load().omp_triad(key, n, s, _p(a))
    return a


def spmv(key: int, rows: int, table):
    """y (fp64), per-row sum |a x|, and row_ptr (int64)."""
    table = np.ascontiguousarray(table, dtype=np.uint64)
    y = np.empty(rows, dtype=np.float64)
    mag = np.empty(rows, dtype=np.float64)
    ptr = np.empty(rows + 1, dtype=np.int64)
    _load().omp_spmv(key, rows, _p(table), _p(y), _p(mag), _p(ptr))
    return y, mag, ptr


def gemm(key: int, m: int, n: int, k: int) -> np.ndarray:
    """C = A B^T in fp64 of the bf16-rounded inputs (M x N)."""
    a = np.empty((m, k), dtype=np.float64)
    b = np.empty((n, k), dtype=np.float64)
    _load().omp_gemm_operand(key, 1, m, k, _p(a))
    _load().omp_gemm_operand(key, 2, n, k, _p(b))
    return a @ b.T

"""The paper's plain CPU method (recursive tensor functions over stride
iterators, Secs. 5.1-5.2), restated as plain C++ in ``recursive.cpp`` and
parallelised over its outermost recursion level with OpenMP.

A timed CPU baseline for ``bench.py``: it shares no code with the GPU library
or with the FP64 oracle.  Tensors are memory buffers in storage order with
extents ``n`` and strides ``w`` (elements); modes ``q`` are 1-based as in the
paper's equations.  Every function computes only the first ``count`` indices
of the highest free mode, so a bounded sample of a call can be timed.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recursive.cpp")
_LIB_PATH = os.path.join(_HERE, "librecursive.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compiles recursive.cpp (g++ -O3 -fopenmp, no host-specific flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cxx = shutil.which("g++") or "g++"
    subprocess.run([cxx, "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.cm_threads.argtypes = [ctypes.c_int]
            lib.cm_transform_f32.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _f32p, _i64p,
                                             _f32p, _i64p, _f32p, _i64p, ctypes.c_int64,
                                             ctypes.c_int]
            lib.cm_ttv_f32.argtypes = [ctypes.c_int, _i64p, _f32p, _i64p, ctypes.c_int, _f32p,
                                       _f32p, _i64p, ctypes.c_int64, ctypes.c_int]
            lib.cm_ttm_f32.argtypes = [ctypes.c_int, _i64p, _f32p, _i64p, ctypes.c_int, _f32p,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _f32p,
                                       _i64p, ctypes.c_int64, ctypes.c_int]
            _lib = lib
        return _lib


def _i64(seq) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int64).reshape(-1))


def _f32(a: np.ndarray):
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError("FP32 contiguous buffers only")
    return a.ctypes.data_as(_f32p)


def threads(request: int = 0) -> int:
    """OpenMP threads the parallel level uses (0 keeps the default)."""
    return int(_load().cm_threads(int(request)))


def _highest_free(p: int, q: int) -> int:
    return p - 2 if q == p else p - 1      # 0-based mode index


def ttv(A, n, wA, q, b, C, wC_by_A, count=None, nthreads=0):
    """C = A x_q b (Eq. 24) into the buffer C; wC_by_A gives C's stride for
    each mode of A (the entry of mode q is ignored)."""
    p = len(n)
    top = _highest_free(p, q)
    count = int(n[top]) if count is None else int(count)
    nn, wa, wc = _i64(n), _i64(wA), _i64(wC_by_A)
    rc = _load().cm_ttv_f32(p, nn.ctypes.data_as(_i64p), _f32(A), wa.ctypes.data_as(_i64p), q - 1,
                            _f32(b), _f32(C), wc.ctypes.data_as(_i64p), count, int(nthreads))
    if rc:
        raise ValueError("cm_ttv_f32 rejected its arguments")


def ttm(A, n, wA, q, B, J, ldb_row, ldb_col, C, wC, count=None, nthreads=0):
    """C = A x_q B (Eq. 25), B(j, k) at B[j*ldb_row + k*ldb_col]; C has A's
    modes with extent J in mode q and strides wC."""
    p = len(n)
    top = _highest_free(p, q)
    count = int(n[top]) if count is None else int(count)
    nn, wa, wc = _i64(n), _i64(wA), _i64(wC)
    rc = _load().cm_ttm_f32(p, nn.ctypes.data_as(_i64p), _f32(A), wa.ctypes.data_as(_i64p), q - 1,
                            _f32(B), int(J), int(ldb_row), int(ldb_col), _f32(C),
                            wc.ctypes.data_as(_i64p), count, int(nthreads))
    if rc:
        raise ValueError("cm_ttm_f32 rejected its arguments")


def transform(op, A, wA, B, wB, C, wC, n, count=None, nthreads=0):
    """C = A op B (Eq. 23; op 0..3 = + - * /) with each operand in its own
    layout, over the first `count` indices of the last mode."""
    p = len(n)
    count = int(n[p - 1]) if count is None else int(count)
    nn, wa, wb, wc = _i64(n), _i64(wA), _i64(wB), _i64(wC)
    rc = _load().cm_transform_f32(p, nn.ctypes.data_as(_i64p), int(op), _f32(A),
                                  wa.ctypes.data_as(_i64p), _f32(B), wb.ctypes.data_as(_i64p),
                                  _f32(C), wc.ctypes.data_as(_i64p), count, int(nthreads))
    if rc:
        raise ValueError("cm_transform_f32 rejected its arguments")

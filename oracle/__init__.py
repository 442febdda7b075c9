"""FP64 CPU oracle for ttv, ttm and entrywise operations (arXiv 1711.10912).

TEST INFRASTRUCTURE ONLY.  The oracle is the independent checker of the CUDA
path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it.  The product package never
imports it, and it imports nothing from the product package.

The arithmetic lives in ``tl_oracle.c`` (plain nested loops in IEEE double,
each function citing the section and equation of the paper it follows).  This
module compiles that file with gcc on first use and marshals numpy buffers to
it.  Tensors are passed as *memory buffers* (1-D arrays in storage order) plus
extents ``n`` and strides ``w`` in elements, exactly the (p, n, pi, w, data)
description of the paper's Sec. 3.1; FP32 inputs are widened to FP64, which is
exact.

Parity status of each function (how it is pinned, see tests/test_oracle_*.py):
  strides, lam, view     pinned by the paper's worked examples, the closed
                         forms of Eqs. 15-16, numpy's own memory layouts and a
                         brute-force bijection check over all layouts.
  ttv, ttv_at            pinned by numpy.tensordot, the p=2 vector-matrix
                         special case, unit-vector slices, all-ones sums,
                         layout invariance and the paper's output shapes.
  ttm, ttm_at            pinned by identity / permutation matrices, J=1 == ttv,
                         the p=2 matrix product, mode commutation, tensordot.
  entrywise              pinned by numpy elementwise ops on logical arrays.
  norm, rel_error        pinned by numpy.linalg.norm and closed forms.
  ttvs, ttms             compositions of ttv / ttm; pinned by numpy einsum, a
                         rank-1 closed form and order independence.
  hopm                   pinned by one-sweep convergence on rank-1 tensors
                         (lambda = sigma) and by p = 2 power iteration against
                         numpy's largest singular value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtl_oracle.so")
_lock = threading.Lock()
_lib = None

OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_COPY, OP_SCALE = range(6)

_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)


def compile_source(src: str, out: str) -> str:
    """Compiles an oracle C source with plain gcc (no flags that change
    floating-point semantics: no -ffast-math, FMA contraction off)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compiles tl_oracle.c into libtl_oracle.so next to it."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


def _bind(path: str):
    """Loads a compiled oracle library and declares its C signatures."""
    lib = ctypes.CDLL(path)
    lib.orc_strides.argtypes = [ctypes.c_uint32, _i64p, _u32p, _i64p]
    lib.orc_strides.restype = ctypes.c_int
    lib.orc_lambda.argtypes = [ctypes.c_uint32, _i64p, _i64p, _i64p]
    lib.orc_lambda.restype = ctypes.c_int64
    lib.orc_view.argtypes = [ctypes.c_uint32, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
                             _i64p, _i64p, _i64p]
    lib.orc_view.restype = ctypes.c_int
    lib.orc_ttv.argtypes = [ctypes.c_uint32, _i64p, ctypes.c_uint32, _f64p, _i64p,
                            _f64p, ctypes.c_int64, _f64p, _i64p, ctypes.c_int, ctypes.c_int]
    lib.orc_ttv.restype = ctypes.c_int
    lib.orc_ttv_at.argtypes = [ctypes.c_uint32, _i64p, ctypes.c_uint32, _f64p, _i64p,
                               _f64p, ctypes.c_int64, _i64p, ctypes.c_int64, _f64p, ctypes.c_int]
    lib.orc_ttv_at.restype = ctypes.c_int
    lib.orc_ttm.argtypes = [ctypes.c_uint32, _i64p, ctypes.c_uint32, _f64p, _i64p,
                            _f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                            _f64p, _i64p, ctypes.c_int, ctypes.c_int]
    lib.orc_ttm.restype = ctypes.c_int
    lib.orc_ttm_at.argtypes = [ctypes.c_uint32, _i64p, ctypes.c_uint32, _f64p, _i64p,
                               _f64p, ctypes.c_int64, ctypes.c_int64, _i64p, ctypes.c_int64,
                               _f64p, ctypes.c_int]
    lib.orc_ttm_at.restype = ctypes.c_int
    lib.orc_entrywise.argtypes = [ctypes.c_int, ctypes.c_uint32, _i64p, _f64p, _i64p,
                                  _f64p, _i64p, ctypes.c_double, _f64p, _i64p]
    lib.orc_entrywise.restype = ctypes.c_int
    lib.orc_transpose.argtypes = [ctypes.c_uint32, _i64p, _f64p, _i64p, _u32p, _f64p, _i64p]
    lib.orc_transpose.restype = ctypes.c_int
    lib.orc_ttt.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                            _i64p, _f64p, _i64p, _u32p, _i64p, _f64p, _i64p, _u32p,
                            _f64p, _i64p, ctypes.c_int, ctypes.c_int]
    lib.orc_ttt.restype = ctypes.c_int
    lib.orc_norm.argtypes = [ctypes.c_uint32, _i64p, _f64p, _i64p, ctypes.c_int]
    lib.orc_norm.restype = ctypes.c_double
    lib.orc_rel_error.argtypes = [ctypes.c_uint32, _i64p, _f64p, _i64p, _f64p, _i64p]
    lib.orc_rel_error.restype = ctypes.c_double
    return lib


def _i64(seq) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int64).reshape(-1))


def _u32(seq) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.uint32).reshape(-1))


def _ptr(a: np.ndarray, ctype, offset: int = 0):
    return ctypes.cast(a.ctypes.data + offset * a.itemsize, ctypes.POINTER(ctype))


def _f64buf(a) -> np.ndarray:
    """Widens a memory buffer to a contiguous float64 copy (exact for f32)."""
    return np.ascontiguousarray(np.asarray(a).reshape(-1), dtype=np.float64)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid arguments (rc={rc})")


# ---------------------------------------------------------------- layout ---

def strides(n, pi=None) -> tuple:
    """Stride tuple of Sec. 3.1 Eq. 14 for extents n and 1-based layout pi."""
    n_ = _i64(n)
    p = len(n_)
    w = np.zeros(p, dtype=np.int64)
    pi_ = None if pi is None else _u32(pi)
    rc = _load().orc_strides(p, _ptr(n_, ctypes.c_int64),
                             None if pi_ is None else _ptr(pi_, ctypes.c_uint32),
                             _ptr(w, ctypes.c_int64))
    _check(rc, "strides")
    return tuple(int(x) for x in w)


def lam(w, i, o=None) -> int:
    """Layout function lambda(w, i, o) of Sec. 3.2 Eq. 17."""
    w_, i_ = _i64(w), _i64(i)
    o_ = None if o is None else _i64(o)
    return int(_load().orc_lambda(len(w_), _ptr(w_, ctypes.c_int64), _ptr(i_, ctypes.c_int64),
                                  None if o_ is None else _ptr(o_, ctypes.c_int64)))


def view(n, w, f, t, l, o=None):
    """View extents, strides and first-element offset (Sec. 3.3 Eqs. 5, 18, 19)."""
    n_, w_, f_, t_, l_ = _i64(n), _i64(w), _i64(f), _i64(t), _i64(l)
    p = len(n_)
    o_ = None if o is None else _i64(o)
    nv = np.zeros(p, dtype=np.int64)
    wv = np.zeros(p, dtype=np.int64)
    g = np.zeros(1, dtype=np.int64)
    rc = _load().orc_view(p, _ptr(n_, ctypes.c_int64), _ptr(w_, ctypes.c_int64),
                          None if o_ is None else _ptr(o_, ctypes.c_int64),
                          _ptr(f_, ctypes.c_int64), _ptr(t_, ctypes.c_int64),
                          _ptr(l_, ctypes.c_int64), _ptr(nv, ctypes.c_int64),
                          _ptr(wv, ctypes.c_int64), _ptr(g, ctypes.c_int64))
    _check(rc, "view")
    return tuple(int(x) for x in nv), tuple(int(x) for x in wv), int(g[0])


def _span(n, w) -> int:
    """Number of buffer elements a strided tensor reaches (max offset + 1)."""
    if any(int(x) == 0 for x in n):
        return 0
    return 1 + sum((int(a) - 1) * int(b) for a, b in zip(n, w))


# ------------------------------------------------------------ operations ---

def ttv(A, n, wA, q, b, incb=1, C=None, wC=None, accumulate=False,
        compensated=False, offA=0):
    """Mode-q tensor-times-vector, Sec. 5.2 Eq. 24, in FP64.

    A is a memory buffer (offset offA to element 0), n its extents, wA its
    strides.  Returns the FP64 output buffer (a fresh first-order buffer when
    C is None, else a float64 copy of C updated in place of the copy)."""
    n_ = _i64(n)
    p = len(n_)
    wA_ = _i64(wA)
    nout = [int(n_[r]) for r in range(p) if r != q - 1]
    if wC is None:
        wC = strides(nout) if p > 1 else ()
    wC_ = _i64(wC)
    Cbuf = np.zeros(max(_span(nout, wC_), 1)) if C is None else _f64buf(C).copy()
    Ab, bb = _f64buf(A), _f64buf(b)
    rc = _load().orc_ttv(p, _ptr(n_, ctypes.c_int64), q, _ptr(Ab, ctypes.c_double, offA),
                         _ptr(wA_, ctypes.c_int64), _ptr(bb, ctypes.c_double), incb,
                         _ptr(Cbuf, ctypes.c_double), _ptr(wC_, ctypes.c_int64),
                         int(accumulate), int(compensated))
    _check(rc, "ttv")
    return Cbuf


def ttv_at(A, n, wA, q, b, out_idx, incb=1, compensated=False, offA=0):
    """Eq. 24 evaluated at the given output multi-indices (cnt x (p-1))."""
    n_ = _i64(n)
    p = len(n_)
    idx = np.ascontiguousarray(np.asarray(out_idx, dtype=np.int64).reshape(-1, p - 1))
    out = np.zeros(idx.shape[0])
    Ab, bb, wA_ = _f64buf(A), _f64buf(b), _i64(wA)
    rc = _load().orc_ttv_at(p, _ptr(n_, ctypes.c_int64), q, _ptr(Ab, ctypes.c_double, offA),
                            _ptr(wA_, ctypes.c_int64), _ptr(bb, ctypes.c_double), incb,
                            _ptr(idx, ctypes.c_int64), idx.shape[0], _ptr(out, ctypes.c_double),
                            int(compensated))
    _check(rc, "ttv_at")
    return out


def ttm(A, n, wA, q, B, J, ldb_row, ldb_col=1, C=None, wC=None, accumulate=False,
        compensated=False, offA=0):
    """Mode-q tensor-times-matrix, Sec. 5.2 Eq. 25, in FP64.

    B(j, k) is B[j*ldb_row + k*ldb_col] for a J x n_q matrix."""
    n_ = _i64(n)
    p = len(n_)
    wA_ = _i64(wA)
    nout = [int(J) if r == q - 1 else int(n_[r]) for r in range(p)]
    if wC is None:
        wC = strides(nout)
    wC_ = _i64(wC)
    Cbuf = np.zeros(max(_span(nout, wC_), 1)) if C is None else _f64buf(C).copy()
    Ab, Bb = _f64buf(A), _f64buf(B)
    rc = _load().orc_ttm(p, _ptr(n_, ctypes.c_int64), q, _ptr(Ab, ctypes.c_double, offA),
                         _ptr(wA_, ctypes.c_int64), _ptr(Bb, ctypes.c_double), int(J),
                         int(ldb_row), int(ldb_col), _ptr(Cbuf, ctypes.c_double),
                         _ptr(wC_, ctypes.c_int64), int(accumulate), int(compensated))
    _check(rc, "ttm")
    return Cbuf


def ttm_at(A, n, wA, q, B, ldb_row, ldb_col, out_idx, compensated=False, offA=0):
    """Eq. 25 evaluated at the given output multi-indices (cnt x p)."""
    n_ = _i64(n)
    p = len(n_)
    idx = np.ascontiguousarray(np.asarray(out_idx, dtype=np.int64).reshape(-1, p))
    out = np.zeros(idx.shape[0])
    Ab, Bb, wA_ = _f64buf(A), _f64buf(B), _i64(wA)
    rc = _load().orc_ttm_at(p, _ptr(n_, ctypes.c_int64), q, _ptr(Ab, ctypes.c_double, offA),
                            _ptr(wA_, ctypes.c_int64), _ptr(Bb, ctypes.c_double), int(ldb_row),
                            int(ldb_col), _ptr(idx, ctypes.c_int64), idx.shape[0],
                            _ptr(out, ctypes.c_double), int(compensated))
    _check(rc, "ttm_at")
    return out


def entrywise(op, n, A, wA, B=None, wB=None, alpha=1.0, C=None, wC=None, offA=0, offB=0):
    """C(i) = A(i) op B(i) (Sec. 5.1 Eq. 23), COPY and SCALE (Eq. 22)."""
    n_ = _i64(n)
    p = len(n_)
    wA_ = _i64(wA)
    wC_ = _i64(strides(n_) if wC is None else wC)
    Cbuf = np.zeros(max(_span(n_, wC_), 1)) if C is None else _f64buf(C).copy()
    Ab = _f64buf(A)
    unary = op in (OP_COPY, OP_SCALE)
    Bb = Ab if unary or B is None else _f64buf(B)
    wB_ = wA_ if unary or wB is None else _i64(wB)
    rc = _load().orc_entrywise(int(op), p, _ptr(n_, ctypes.c_int64),
                               _ptr(Ab, ctypes.c_double, offA), _ptr(wA_, ctypes.c_int64),
                               _ptr(Bb, ctypes.c_double, 0 if unary else offB),
                               _ptr(wB_, ctypes.c_int64), float(alpha),
                               _ptr(Cbuf, ctypes.c_double), _ptr(wC_, ctypes.c_int64))
    _check(rc, "entrywise")
    return Cbuf


def transpose(A, nA, wA, tau, C=None, wC=None, offA=0):
    """C = A^tau (Table 3, transpose): C(i^c) = A(i^a) with i^c_r = i^a_{tau_r}
    and n^c_r = n^a_{tau_r}.  Returns (FP64 buffer of C, C's extents)."""
    nA_ = _i64(nA)
    p = len(nA_)
    tau_ = _u32(tau)
    nc = tuple(int(nA_[int(t) - 1]) for t in tau_)
    wC_ = _i64(strides(nc) if wC is None else wC)
    Cbuf = np.zeros(max(_span(nc, wC_), 1)) if C is None else _f64buf(C).copy()
    Ab, wA_ = _f64buf(A), _i64(wA)
    rc = _load().orc_transpose(p, _ptr(nA_, ctypes.c_int64), _ptr(Ab, ctypes.c_double, offA),
                               _ptr(wA_, ctypes.c_int64), _ptr(tau_, ctypes.c_uint32),
                               _ptr(Cbuf, ctypes.c_double), _ptr(wC_, ctypes.c_int64))
    _check(rc, "transpose")
    return Cbuf, nc


def ttt_shape(nA, nB, q, phi, psi):
    """Output extents of the (q, phi, psi)-mode product (Sec. 5.2)."""
    r, s = len(nA) - q, len(nB) - q
    return tuple(int(nA[phi[k] - 1]) for k in range(r)) + \
        tuple(int(nB[psi[k] - 1]) for k in range(s))


def ttt(A, nA, wA, phi, B, nB, wB, psi, q, C=None, wC=None, accumulate=False,
        compensated=False, offA=0, offB=0):
    """(q, phi, psi)-mode tensor-tensor multiplication (Sec. 5.2) in FP64.
    phi / psi are 1-based; their first r / s entries order C's modes and
    their last q entries pair the contracted modes.  Returns (FP64 buffer of
    C, C's extents); an order-0 result is a one-element buffer."""
    nA_, nB_ = _i64(nA), _i64(nB)
    q = int(q)
    r, s = len(nA_) - q, len(nB_) - q
    if r < 0 or s < 0 or len(phi) != len(nA_) or len(psi) != len(nB_):
        raise ValueError("phi / psi must have q+r / q+s entries")
    nc = ttt_shape(nA_, nB_, q, list(phi), list(psi))
    wC_ = _i64((strides(nc) if nc else ()) if wC is None else wC)
    Cbuf = np.zeros(max(_span(nc, wC_) if nc else 1, 1)) if C is None else _f64buf(C).copy()
    Ab, Bb = _f64buf(A), _f64buf(B)
    wA_, wB_ = _i64(wA), _i64(wB)
    phi_, psi_ = _u32(phi), _u32(psi)
    rc = _load().orc_ttt(q, r, s, _ptr(nA_, ctypes.c_int64), _ptr(Ab, ctypes.c_double, offA),
                         _ptr(wA_, ctypes.c_int64), _ptr(phi_, ctypes.c_uint32),
                         _ptr(nB_, ctypes.c_int64), _ptr(Bb, ctypes.c_double, offB),
                         _ptr(wB_, ctypes.c_int64), _ptr(psi_, ctypes.c_uint32),
                         _ptr(Cbuf, ctypes.c_double),
                         _ptr(wC_ if len(wC_) else _i64([0]), ctypes.c_int64),
                         int(accumulate), int(compensated))
    _check(rc, "ttt")
    return Cbuf, nc


def norm(A, n, wA, compensated=True, offA=0) -> float:
    """Frobenius norm (Table 3, norm) in FP64."""
    n_, wA_, Ab = _i64(n), _i64(wA), _f64buf(A)
    return float(_load().orc_norm(len(n_), _ptr(n_, ctypes.c_int64),
                                  _ptr(Ab, ctypes.c_double, offA), _ptr(wA_, ctypes.c_int64),
                                  int(compensated)))


def rel_error(X, wX, R, wR, n) -> float:
    """||X - R||_F / ||R||_F with each tensor in its own layout."""
    n_, wX_, wR_ = _i64(n), _i64(wX), _i64(wR)
    Xb, Rb = _f64buf(X), _f64buf(R)
    return float(_load().orc_rel_error(len(n_), _ptr(n_, ctypes.c_int64),
                                       _ptr(Xb, ctypes.c_double), _ptr(wX_, ctypes.c_int64),
                                       _ptr(Rb, ctypes.c_double), _ptr(wR_, ctypes.c_int64)))


# ------------------------------------------------- sequences and HOPM ---

def ttvs(A, n, wA, modes, vecs, offA=0):
    """Tensor times several vectors (Sec. 5.2 Table 3, times_vectors): A is
    contracted with vecs[j] along the distinct 1-based modes[j], applying the
    vectors from the last listed to the first (the order the paper states for
    times_vectors, so the remaining mode numbers stay valid).  Each step is
    one oracle ttv (Eq. 24) into a dense first-order FP64 intermediate.
    Returns (buffer, extents of the remaining modes in order)."""
    n = [int(x) for x in n]
    modes = [int(m) for m in modes]
    if len(set(modes)) != len(modes) or any(m < 1 or m > len(n) for m in modes):
        raise ValueError("modes must be distinct and within 1..p")
    if len(modes) >= len(n):
        raise ValueError("a sequence of ttv (Eq. 24, order >= 2) leaves at least one mode")
    cur, cur_n, cur_w, cur_off = A, list(n), list(wA), offA
    alive = list(range(1, len(n) + 1))          # original mode numbers still present
    for m, v in reversed(list(zip(modes, vecs))):
        q = alive.index(m) + 1
        out = ttv(cur, cur_n, cur_w, q, v, offA=cur_off)
        del cur_n[q - 1]
        alive.remove(m)
        cur, cur_w, cur_off = out, list(strides(cur_n)) if cur_n else [], 0
    return cur, tuple(cur_n)


def ttms(A, n, wA, modes, mats, offA=0):
    """Tensor times several matrices (Sec. 5.2 Table 3, times_matrices):
    mats[j] is J_j x n_{modes[j]} (row-major); applied from the last listed to
    the first, each step one oracle ttm (Eq. 25) into a dense first-order
    FP64 intermediate.  Returns (buffer, output extents)."""
    cur, cur_n, cur_w, cur_off = A, [int(x) for x in n], list(wA), offA
    for m, M in reversed(list(zip(modes, mats))):
        M = np.asarray(M)
        J, K = M.shape
        if K != cur_n[m - 1]:
            raise ValueError("matrix columns must equal the mode's extent")
        out = ttm(cur, cur_n, cur_w, m, M.reshape(-1), J, K, 1, offA=cur_off)
        cur_n[m - 1] = J
        cur, cur_w, cur_off = out, list(strides(cur_n)), 0
    return cur, tuple(cur_n)


def hopm(A, n, wA, u0, K):
    """Higher-order power method for the best rank-1 approximation, following
    the paper's listing in Sec. 5.2 (after De Lathauwer et al.): K sweeps; in
    each, for r = 1..p, u_r <- A times all vectors except u_r (times_vectors
    with mode r excluded), lambda_r <- ||u_r||, u_r <- u_r / lambda_r.
    Returns (list of u vectors, list of lambdas), all FP64."""
    p = len(n)
    u = [np.asarray(x, dtype=np.float64).copy() for x in u0]
    lam = [0.0] * p
    for _ in range(int(K)):
        for r in range(1, p + 1):
            others = [m for m in range(1, p + 1) if m != r]
            vec, rest = ttvs(A, n, wA, others, [u[m - 1] for m in others])
            assert rest == (int(n[r - 1]),)
            lam[r - 1] = norm(vec, rest, (1,))
            u[r - 1] = vec / lam[r - 1]
    return u, lam

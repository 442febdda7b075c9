"""Python binding of libtlgb.so, the GB300 (sm_103a) ttv / ttm / entrywise library.

Argument marshalling only: each ``tl_*`` function here has the name, argument
order and return code of its C counterpart in ``include/tlgb.h``; every step of
the computation runs in the library's CUDA kernels.  There is no fallback: if
the shared library is missing, every call raises ImportError.
Build it with ``python -m paper_1711_10912_gb300.build`` (or
``__graft_entry__.build()``).

Tensors are passed as :class:`Desc` objects built from a device address (or a
torch tensor's ``data_ptr()``), the extents ``n``, an optional 1-based layout
tuple ``pi`` and optional strides ``w`` in elements, i.e. the (p, n, pi, w)
description of the TLib paper's Sec. 3.1.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# TL_LIBRARY selects another build of the library (the bounds-checked
# libtlgb_checked.so, for instance); the default is the product build.
LIB_PATH = os.environ.get("TL_LIBRARY") or os.path.join(_HERE, "libtlgb.so")


class _MissingLibrary:
    """Stands in for the library when libtlgb.so has not been built: every
    use raises, so nothing can silently run without the CUDA kernels."""

    def __getattr__(self, name):
        raise ImportError(
            f"libtlgb.so not found at {LIB_PATH}: build it with "
            "`python -m paper_1711_10912_gb300.build` (there is no CPU fallback)")


_lib = _MissingLibrary()

TL_OK, TL_EINVAL, TL_EUNSUPPORTED, TL_ENOMEM, TL_ECUDA, TL_ETIMEOUT, TL_ECANCELED = \
    0, -1, -2, -3, -4, -5, -6
TL_PENDING = 1
TL_EBOUNDS = -7
TL_F32, TL_F64 = 0, 1
TL_P_DEFAULT, TL_P_F64, TL_P_F32, TL_P_TF32, TL_P_BF16, TL_P_BF16X3 = range(6)
TL_ADD, TL_SUB, TL_MUL, TL_DIV, TL_COPY, TL_SCALE = range(6)
TL_OP_TTV, TL_OP_TTM, TL_OP_ENTRYWISE = range(3)
TL_CTX_PERSISTENT, TL_CTX_GRAPH = 1, 2
TL_BATCH_GRAPH, TL_BATCH_TUNE = 1, 2
(TL_BV_TTV_COL, TL_BV_TTV_ROW4, TL_BV_TTV_ROW8, TL_BV_TTV_ROW32, TL_BV_TTM_32, TL_BV_TTM_64,
 TL_BV_EW, TL_BV_TTM_SMALL, TL_BV_TTV_VEC) = range(9)

_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class tl_tensor(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint32), ("dtype", ctypes.c_int32), ("n", _i64p),
                ("pi", _u32p), ("w", _i64p), ("data", ctypes.c_void_p)]


class tl_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("entry_op", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("accumulate", ctypes.c_int32),
                ("q", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("J", ctypes.c_int64), ("ldb_row", ctypes.c_int64), ("ldb_col", ctypes.c_int64),
                ("incb", ctypes.c_int64), ("alpha", ctypes.c_double), ("vec", ctypes.c_void_p),
                ("A", tl_tensor), ("B", tl_tensor), ("C", tl_tensor)]


class TLError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {tl_strerror(code)} ({code})")
        self.code = code


def _dtype_code(dtype) -> int:
    s = str(dtype)
    if s.endswith("float32") or s in ("f32", "float32"):
        return TL_F32
    if s.endswith("float64") or s in ("f64", "float64"):
        return TL_F64
    raise ValueError(f"unsupported dtype {dtype}")


class Desc:
    """Owns the ctypes arrays of one tl_tensor descriptor."""

    def __init__(self, data, n, pi=None, w=None, dtype=None):
        if hasattr(data, "data_ptr"):
            if dtype is None:
                dtype = data.dtype
            self._keep = data
            addr = data.data_ptr()
        else:
            addr = int(data)
        if dtype is None:
            raise ValueError("dtype required for a raw address")
        self.n_arr = (ctypes.c_int64 * max(len(n), 1))(*[int(x) for x in n])
        self.pi_arr = None if pi is None else (ctypes.c_uint32 * len(pi))(*[int(x) for x in pi])
        self.w_arr = None if w is None else (ctypes.c_int64 * len(w))(*[int(x) for x in w])
        self.n = tuple(int(x) for x in n)
        self.pi = None if pi is None else tuple(int(x) for x in pi)
        self.w = None if w is None else tuple(int(x) for x in w)
        self.s = tl_tensor(len(n), _dtype_code(dtype),
                           ctypes.cast(self.n_arr, _i64p),
                           None if self.pi_arr is None else ctypes.cast(self.pi_arr, _u32p),
                           None if self.w_arr is None else ctypes.cast(self.w_arr, _i64p),
                           ctypes.c_void_p(addr))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _addr(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s) -> ctypes.c_void_p:
    if s is None:
        return ctypes.c_void_p(0)
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def _ref(d):
    return None if d is None else d.ref


# ------------------------------------------------------------ signatures ---
_T = ctypes.POINTER(tl_tensor)


def load_library():
    """Loads libtlgb.so and declares the C signatures (called at import when
    the library exists, and again after a build)."""
    global _lib
    if not os.path.exists(LIB_PATH):
        _lib = _MissingLibrary()
        return _lib
    lib = ctypes.CDLL(LIB_PATH)
    _declare(lib)
    _lib = lib
    return lib


def _declare(_lib):
    _lib.tl_ttv.argtypes = [_T, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, _T,
                            ctypes.c_int32, ctypes.c_void_p]
    _lib.tl_ttv_noalloc.argtypes = [_T, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, _T,
                                     ctypes.c_int32, ctypes.c_void_p]
    _lib.tl_ttm.argtypes = [_T, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_uint32, _T, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    _lib.tl_entrywise.argtypes = [ctypes.c_int32, _T, _T, ctypes.c_double, _T, ctypes.c_void_p]
    _lib.tl_norm.argtypes = [_T, ctypes.c_void_p, ctypes.c_void_p]
    _lib.tl_rel_error.argtypes = [_T, _T, ctypes.c_void_p, ctypes.c_void_p]
    _lib.tl_launch_count.restype = ctypes.c_uint64
    _lib.tl_device_status.argtypes = [ctypes.c_void_p]
    _lib.tl_strerror.argtypes = [ctypes.c_int]
    _lib.tl_strerror.restype = ctypes.c_char_p
    _lib.tl_plan_describe.argtypes = [ctypes.c_int32, _T, _T, ctypes.c_uint32, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_int32, _T, ctypes.c_char_p,
                                      ctypes.c_size_t]
    _lib.tl_ctx_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_void_p)]
    _lib.tl_ctx_destroy.argtypes = [ctypes.c_void_p]
    _lib.tl_batch_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(tl_op), ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_uint64)]
    _lib.tl_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_double)]
    _lib.tl_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    _lib.tl_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    _lib.tl_ctx_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                  ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    _lib.tl_batch_create.argtypes = [ctypes.POINTER(tl_op), ctypes.c_size_t, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    _lib.tl_batch_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    _lib.tl_batch_destroy.argtypes = [ctypes.c_void_p]
    _lib.tl_batch_describe.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    _lib.tl_batch_set_variant.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int64, ctypes.c_void_p]
    _lib.tl_selftest_wait_timeout.argtypes = [ctypes.c_double, ctypes.c_void_p]
    _lib.tl_bounds_checked.restype = ctypes.c_int
    _lib.tl_fma_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    _lib.tl_ttvs.argtypes = [_T, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint32),
                             ctypes.c_uint32, _T, ctypes.c_void_p]
    _lib.tl_ttms.argtypes = [_T, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32, _T, ctypes.c_int32,
                             ctypes.c_void_p]
    _lib.tl_transpose.argtypes = [_T, ctypes.POINTER(ctypes.c_uint32), _T, ctypes.c_void_p]
    _lib.tl_ttt.argtypes = [_T, ctypes.POINTER(ctypes.c_uint32), _T,
                            ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32, _T, ctypes.c_int32,
                            ctypes.c_int32, ctypes.c_void_p]
    _lib.tl_view.argtypes = [_T, _i64p, _i64p, _i64p, _T, _i64p, _i64p]
    _lib.tl_hopm.argtypes = [_T, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_uint32,
                             ctypes.c_void_p]


load_library()


# ------------------------------------------------ C-named entry points -----

def tl_version() -> int:
    return _lib.tl_version()


def tl_launch_count() -> int:
    return int(_lib.tl_launch_count())


def tl_device_status(stream=None) -> int:
    return _lib.tl_device_status(_stream(stream))


def tl_strerror(code: int) -> str:
    return _lib.tl_strerror(int(code)).decode()


def tl_ttv(A: Desc, b, incb: int, q: int, C: Desc, accumulate: int = 0, stream=None) -> int:
    return _lib.tl_ttv(A.ref, _addr(b), int(incb), int(q), C.ref, int(accumulate), _stream(stream))


def tl_ttv_noalloc(A: Desc, b, incb: int, q: int, C: Desc, accumulate: int = 0,
                   stream=None) -> int:
    return _lib.tl_ttv_noalloc(A.ref, _addr(b), int(incb), int(q), C.ref, int(accumulate),
                               _stream(stream))


TL_TTV_NOALLOC_SCRATCH_BYTES = 4 << 20


def tl_ttm(A: Desc, B, J: int, ldb_row: int, ldb_col: int, q: int, C: Desc,
           precision: int = TL_P_DEFAULT, accumulate: int = 0, stream=None) -> int:
    return _lib.tl_ttm(A.ref, _addr(B), int(J), int(ldb_row), int(ldb_col), int(q), C.ref,
                       int(precision), int(accumulate), _stream(stream))


def tl_entrywise(op: int, A: Desc, B, alpha: float, C: Desc, stream=None) -> int:
    return _lib.tl_entrywise(int(op), A.ref, _ref(B), float(alpha), C.ref, _stream(stream))


def _ptr_array(xs):
    return (ctypes.c_void_p * max(len(xs), 1))(*[_addr(x) for x in xs])


def tl_ttvs(A: Desc, vecs, modes, C: Desc, stream=None) -> int:
    m = (ctypes.c_uint32 * max(len(modes), 1))(*[int(x) for x in modes])
    return _lib.tl_ttvs(A.ref, _ptr_array(vecs), m, len(modes), C.ref, _stream(stream))


def tl_ttms(A: Desc, mats, J, modes, C: Desc, precision: int = TL_P_DEFAULT, stream=None) -> int:
    m = (ctypes.c_uint32 * max(len(modes), 1))(*[int(x) for x in modes])
    j = (ctypes.c_int64 * max(len(J), 1))(*[int(x) for x in J])
    return _lib.tl_ttms(A.ref, _ptr_array(mats), j, m, len(modes), C.ref, int(precision),
                        _stream(stream))


def tl_hopm(A: Desc, u, lam, K: int, stream=None) -> int:
    return _lib.tl_hopm(A.ref, _ptr_array(u), _addr(lam), int(K), _stream(stream))


def _u32_array(xs):
    return (ctypes.c_uint32 * max(len(xs), 1))(*[int(x) for x in xs])


def tl_transpose(A: Desc, tau, C: Desc, stream=None) -> int:
    return _lib.tl_transpose(A.ref, _u32_array(tau), C.ref, _stream(stream))


def tl_ttt(A: Desc, phi, B: Desc, psi, q: int, C: Desc, precision: int = TL_P_DEFAULT,
           accumulate: int = 0, stream=None) -> int:
    return _lib.tl_ttt(A.ref, _u32_array(phi), B.ref, _u32_array(psi), int(q), C.ref,
                       int(precision), int(accumulate), _stream(stream))


def tl_norm(A: Desc, result, stream=None) -> int:
    return _lib.tl_norm(A.ref, _addr(result), _stream(stream))


def tl_rel_error(X: Desc, R: Desc, result, stream=None) -> int:
    return _lib.tl_rel_error(X.ref, R.ref, _addr(result), _stream(stream))


def tl_view(A: Desc, f, t, l):
    """Descriptor of the view (f, t, l) of A (Sec. 3.3); returns (code, Desc)."""
    p = len(A.n)
    fa, ta, la = (ctypes.c_int64 * p)(*f), (ctypes.c_int64 * p)(*t), (ctypes.c_int64 * p)(*l)
    nv, wv = (ctypes.c_int64 * p)(), (ctypes.c_int64 * p)()
    V = tl_tensor()
    rc = _lib.tl_view(A.ref, fa, ta, la, ctypes.byref(V), nv, wv)
    if rc != TL_OK:
        return rc, None
    D = Desc(int(V.data or 0), tuple(nv), w=tuple(wv),
             dtype="f64" if V.dtype == TL_F64 else "f32")
    D._keep = getattr(A, "_keep", None)
    return rc, D


def tl_plan_describe(op: int, A: Desc, B, q: int, J: int, precision: int, entry_op: int,
                     C: Desc):
    """Returns (code, json-string) for the plan the entry point would run."""
    buf = ctypes.create_string_buffer(4096)
    rc = _lib.tl_plan_describe(int(op), A.ref, _ref(B), int(q), int(J), int(precision),
                               int(entry_op), C.ref, buf, len(buf))
    return rc, buf.value.decode()


def tl_ctx_create(budget_bytes: int, streams: int = 2, flags: int = 0):
    out = ctypes.c_void_p()
    rc = _lib.tl_ctx_create(int(budget_bytes), int(streams), int(flags), ctypes.byref(out))
    return rc, out


def tl_ctx_destroy(ctx) -> int:
    return _lib.tl_ctx_destroy(ctx)


def tl_batch_submit(ctx, ops) -> tuple:
    arr = (tl_op * len(ops))(*ops)
    ticket = ctypes.c_uint64()
    rc = _lib.tl_batch_submit(ctx, arr, len(ops), ctypes.byref(ticket))
    return rc, ticket.value


def tl_poll(ctx, ticket: int) -> tuple:
    st, lat = ctypes.c_int32(), ctypes.c_double()
    rc = _lib.tl_poll(ctx, int(ticket), ctypes.byref(st), ctypes.byref(lat))
    return rc, st.value, lat.value


def tl_wait(ctx, ticket: int, timeout_ms: float = 60000.0) -> tuple:
    st, lat = ctypes.c_int32(), ctypes.c_double()
    rc = _lib.tl_wait(ctx, int(ticket), float(timeout_ms), ctypes.byref(st), ctypes.byref(lat))
    return rc, st.value, lat.value


def tl_cancel(ctx, ticket: int) -> int:
    return _lib.tl_cancel(ctx, int(ticket))


def tl_ctx_stats(ctx) -> tuple:
    m, b, c = ctypes.c_size_t(), ctypes.c_uint64(), ctypes.c_uint64()
    rc = _lib.tl_ctx_stats(ctx, ctypes.byref(m), ctypes.byref(b), ctypes.byref(c))
    return rc, m.value, b.value, c.value


def tl_batch_create(ops, flags: int = 0, stream=None) -> tuple:
    arr = (tl_op * max(len(ops), 1))(*ops)
    out = ctypes.c_void_p()
    rc = _lib.tl_batch_create(arr, len(ops), int(flags), _stream(stream), ctypes.byref(out))
    return rc, out


def tl_batch_run(batch, stream=None) -> int:
    return _lib.tl_batch_run(batch, _stream(stream))


def tl_batch_destroy(batch) -> int:
    return _lib.tl_batch_destroy(batch)


def tl_bounds_checked() -> int:
    """1 if the loaded library is the bounds-checked debug build."""
    return int(_lib.tl_bounds_checked())


def tl_fma_peak_probe(dtype: int, iters: int, sink, stream=None) -> tuple:
    """Enqueues the FMA throughput probe; returns (rc, flops it performs)."""
    f = ctypes.c_double(0.0)
    rc = _lib.tl_fma_peak_probe(int(dtype), int(iters), _addr(sink), ctypes.byref(f),
                                _stream(stream))
    return rc, f.value


def tl_batch_describe(batch) -> tuple:
    buf = ctypes.create_string_buffer(1024)
    rc = _lib.tl_batch_describe(batch, buf, len(buf))
    return rc, buf.value.decode()


def tl_batch_set_variant(batch, kind: int, variant: int, unit: int, stream=None) -> int:
    return _lib.tl_batch_set_variant(batch, int(kind), int(variant), int(unit), _stream(stream))


def tl_selftest_wait_timeout(limit_us: float, stream=None) -> int:
    return _lib.tl_selftest_wait_timeout(float(limit_us), _stream(stream))


def make_op(kind: int, A: Desc, C: Desc, q: int = 0, vec=None, B: Desc = None, J: int = 0,
            ldb_row: int = 0, ldb_col: int = 1, incb: int = 1, precision: int = TL_P_DEFAULT,
            accumulate: int = 0, entry_op: int = TL_ADD, alpha: float = 1.0) -> tl_op:
    """Fills a tl_op; the Desc objects must outlive every use of the op."""
    o = tl_op()
    o.kind, o.entry_op, o.precision, o.accumulate = int(kind), int(entry_op), int(precision), \
        int(accumulate)
    o.q, o.J, o.ldb_row, o.ldb_col, o.incb, o.alpha = int(q), int(J), int(ldb_row), int(ldb_col), \
        int(incb), float(alpha)
    o.vec = ctypes.c_void_p(_addr(vec))
    o.A = A.s
    o.C = C.s
    if B is not None:
        o.B = B.s
    return o


def check(rc: int, what: str = "tl call") -> None:
    """Raises TLError for a negative return code."""
    if rc < 0:
        raise TLError(rc, what)

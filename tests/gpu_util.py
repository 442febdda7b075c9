"""Helpers for the GPU parity tests: move logical numpy arrays to the device in
a given layout, call the C ABI through the binding, and bring results back as
logical arrays.  The reference values always come from the FP64 oracle."""
import numpy as np
import torch

import oracle
import synth

TOL = {"f64": 1e-12, "f32": 1e-5}          # relative Frobenius error bounds
NP = {"f64": np.float64, "f32": np.float32}
TORCH = {"f64": torch.float64, "f32": torch.float32}


def to_dev(mem, dev, dtype):
    return torch.from_numpy(np.ascontiguousarray(mem, dtype=NP[dtype])).to(dev)


def put(X, pi, dev, dtype):
    """Device buffer holding logical array X in dense layout pi."""
    return to_dev(synth.to_memory(np.asarray(X, dtype=NP[dtype]), pi), dev, dtype)


def get(t, n, pi):
    return synth.from_memory(t.detach().cpu().numpy(), n, pi)


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(ref.ravel())
    e = np.linalg.norm((got - ref).ravel())
    return e / d if d > 0 else e


def ttv_case(tl, dev, X, q, b, pi_a, pi_c, dtype, accumulate=False, C0=None, incb=1):
    """Runs tl_ttv on logical inputs; returns (gpu logical, oracle logical)."""
    n = X.shape
    p = len(n)
    nout = tuple(x for r, x in enumerate(n) if r != q - 1)
    Xd = np.asarray(X, dtype=NP[dtype])
    bd = np.asarray(b, dtype=NP[dtype])
    A = put(Xd, pi_a, dev, dtype)
    bbuf = np.zeros((len(bd) - 1) * incb + 1, dtype=NP[dtype])
    bbuf[::incb] = bd
    bt = to_dev(bbuf, dev, dtype)
    C0d = np.zeros(nout, dtype=NP[dtype]) if C0 is None else np.asarray(C0, dtype=NP[dtype])
    C = put(C0d, pi_c, dev, dtype)
    rc = tl.tl_ttv(tl.Desc(A, n, pi_a), bt, incb, q, tl.Desc(C, nout, pi_c), int(accumulate))
    tl.check(rc, "tl_ttv")
    torch.cuda.synchronize()
    got = get(C, nout, pi_c)
    wA = oracle.strides(n, pi_a)
    wC = oracle.strides(nout, pi_c)
    ref = oracle.ttv(synth.to_memory(Xd, pi_a), n, wA, q, bbuf, incb=incb,
                     C=synth.to_memory(C0d, pi_c), wC=wC, accumulate=accumulate)
    return got, synth.from_memory(ref, nout, pi_c)


def ttm_case(tl, dev, X, q, Bm, pi_a, pi_c, dtype, precision=0, accumulate=False, C0=None,
             col_major=False):
    n = X.shape
    J = Bm.shape[0]
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    Xd = np.asarray(X, dtype=NP[dtype])
    Bd = np.asarray(Bm, dtype=NP[dtype])
    A = put(Xd, pi_a, dev, dtype)
    if col_major:
        Bbuf, ldr, ldc = np.ascontiguousarray(Bd.T).reshape(-1), 1, J
    else:
        Bbuf, ldr, ldc = np.ascontiguousarray(Bd).reshape(-1), Bd.shape[1], 1
    Bt = to_dev(Bbuf, dev, dtype)
    C0d = np.zeros(nout, dtype=NP[dtype]) if C0 is None else np.asarray(C0, dtype=NP[dtype])
    C = put(C0d, pi_c, dev, dtype)
    rc = tl.tl_ttm(tl.Desc(A, n, pi_a), Bt, J, ldr, ldc, q, tl.Desc(C, nout, pi_c), precision,
                   int(accumulate))
    tl.check(rc, "tl_ttm")
    torch.cuda.synchronize()
    got = get(C, nout, pi_c)
    wA = oracle.strides(n, pi_a)
    wC = oracle.strides(nout, pi_c)
    ref = oracle.ttm(synth.to_memory(Xd, pi_a), n, wA, q, Bbuf, J, ldr, ldc,
                     C=synth.to_memory(C0d, pi_c), wC=wC, accumulate=accumulate)
    return got, synth.from_memory(ref, nout, pi_c)


def dot_bound(absX, absb, q, eps):
    """Per-element rounding bound of a length-n_q dot product."""
    nq = absX.shape[q - 1]
    return 2 * nq * eps * np.tensordot(absX, absb, axes=([q - 1], [0]))

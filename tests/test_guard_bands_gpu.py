"""Out-of-bounds write detection without a device sanitizer: every output is
placed inside a larger buffer whose guard zones (before, after, and the gaps
of a strided output view) hold canary values; after the call the canaries
must be bit-identical and the output must match the FP64 oracle.  Covers
every kernel path: ttv (row, column, staged rows, split-K), ttm (tiles, short
contractions, split-K, tensor cores in both orientations), entrywise (flat,
TMA tiles, register tiles, rows, generic), transposition, ttt, norm and the
persistent batch."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, TOL, TORCH, put, rel_err, to_dev

gpu = pytest.mark.gpu

GUARD = 4099          # canary elements on each side (odd, to misalign the output too)
CANARY = {"f32": np.float32(-1234.5), "f64": np.float64(-98765.25)}


class Guarded:
    """A device buffer holding an output of extents n as a view with steps
    `t` (gaps between elements hold canaries) and GUARD canaries around it.
    `align` elements of offset keep 16-byte vector paths possible."""

    def __init__(self, dev, dtype, n, t=None, align=True):
        self.dtype = dtype
        self.n = tuple(n)
        self.t = tuple(t) if t else (1,) * len(n)
        self.parent = tuple(x * s for x, s in zip(self.n, self.t))
        size = int(np.prod(self.parent))
        self.off = GUARD + (1 if not align else 0)
        self.off = (self.off + 3) // 4 * 4 if align else self.off
        total = self.off + size + GUARD
        self.buf = torch.full((total,), float(CANARY[dtype]), dtype=TORCH[dtype], device=dev)
        self.wp = oracle.strides(self.parent)
        self.w = tuple(w * s for w, s in zip(self.wp, self.t))
        elem = 8 if dtype == "f64" else 4
        self.ptr = self.buf.data_ptr() + self.off * elem
        # element positions the view owns
        idx = np.indices(self.n).reshape(len(self.n), -1).T
        self.pos = self.off + idx @ np.asarray(self.w, dtype=np.int64)

    def desc(self, tl):
        return tl.Desc(self.ptr, self.n, w=self.w, dtype=self.dtype)

    def check(self):
        if self.buf.is_cuda:
            torch.cuda.synchronize()
        host = self.buf.cpu().numpy()
        mask = np.ones(host.shape[0], dtype=bool)
        mask[self.pos] = False
        bad = np.nonzero(host[mask] != CANARY[self.dtype])[0]
        assert bad.size == 0, f"{bad.size} canaries overwritten"
        # the view's values in logical order (first index fastest, as oracle buffers)
        idx = np.indices(self.n).reshape(len(self.n), -1, order="F").T
        return host[self.off + idx @ np.asarray(self.w, dtype=np.int64)]


def _dense_first(X):
    return synth.to_memory(X, synth.first_order(X.ndim))


@gpu
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n,q,pi,t", [((256, 64, 4), 1, (1, 2, 3), None),      # staged rows
                                      ((37, 20, 9), 2, (2, 3, 1), (1, 2)),     # column, strided C
                                      ((3, 200000), 2, (1, 2), None),          # split-K
                                      ((64, 40, 7), 1, (3, 1, 2), (2, 1))])    # row groups
def test_ttv_guarded(tl, cuda_dev, dtype, n, q, pi, t):
    X = synth.uniform(n, 4800 + q)
    b = synth.uniform((n[q - 1],), 4801 + q)
    A = put(X, pi, cuda_dev, dtype)
    nout = tuple(x for r, x in enumerate(n) if r != q - 1)
    G = Guarded(cuda_dev, dtype, nout, t)
    tl.check(tl.tl_ttv(tl.Desc(A, n, pi), to_dev(b, cuda_dev, dtype), 1, q, G.desc(tl), 0))
    got = G.check()
    ref = oracle.ttv(synth.to_memory(np.asarray(X, NP[dtype]), pi), n, oracle.strides(n, pi), q,
                     np.asarray(b, NP[dtype]))
    assert rel_err(got, ref) <= TOL[dtype]


@gpu
@pytest.mark.parametrize("case", ["tiles", "rows", "splitk", "tc_row", "tc_col"])
def test_ttm_guarded(tl, cuda_dev, case):
    dtype, prec = "f32", 0
    if case == "tiles":
        n, q, J, pi, t, dtype = (129, 67, 33), 1, 70, (1, 2, 3), (1, 2, 1), "f64"
    elif case == "rows":
        n, q, J, pi, t = (300, 5, 17), 2, 21, (2, 1, 3), None
    elif case == "splitk":
        n, q, J, pi, t = (4, 150000), 2, 9, (1, 2), None
    elif case == "tc_row":
        n, q, J, pi, t, prec = (128, 96, 9), 1, 48, (1, 2, 3), None, 5
    else:
        n, q, J, pi, t, prec = (128, 96, 9), 2, 40, (1, 2, 3), None, 5
    X = synth.uniform(n, 4810)
    Bm = synth.uniform((J, n[q - 1]), 4811)
    A = put(X, pi, cuda_dev, dtype)
    nm = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    G = Guarded(cuda_dev, dtype, nm, t)
    tl.check(tl.tl_ttm(tl.Desc(A, n, pi), to_dev(Bm.reshape(-1), cuda_dev, dtype), J, n[q - 1], 1,
                       q, G.desc(tl), prec, 0))
    got = G.check()
    ref = oracle.ttm(synth.to_memory(np.asarray(X, NP[dtype]), pi), n, oracle.strides(n, pi), q,
                     np.asarray(Bm, NP[dtype]).reshape(-1), J, n[q - 1], 1)
    assert rel_err(got, ref) <= (1e-5 if prec else TOL[dtype])


@gpu
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n,pa,pb,op", [((64, 48, 20), (1, 2, 3), (1, 2, 3), 0),   # flat
                                        ((96, 33, 8), (3, 2, 1), (1, 2, 3), 2),    # tiles
                                        ((12, 5, 7, 3), (1, 3, 2, 4), (1, 2, 3, 4), 3),  # rows
                                        ((13, 3, 7, 5, 4), (5, 3, 1, 2, 4), (2, 4, 5, 1, 3), 0)])
def test_entrywise_guarded(tl, cuda_dev, dtype, n, pa, pb, op):
    X = synth.uniform(n, 4820)
    Y = synth.uniform(n, 4821) + 3.0
    A, B = put(X, pa, cuda_dev, dtype), put(Y, pb, cuda_dev, dtype)
    G = Guarded(cuda_dev, dtype, n)          # C dense first-order inside the guard band
    tl.check(tl.tl_entrywise(op, tl.Desc(A, n, pa), tl.Desc(B, n, pb), 1.0, G.desc(tl)))
    got = G.check()
    ref = oracle.entrywise(op, n, synth.to_memory(np.asarray(X, NP[dtype]), pa),
                           oracle.strides(n, pa), synth.to_memory(np.asarray(Y, NP[dtype]), pb),
                           oracle.strides(n, pb))
    np.testing.assert_array_equal(got.astype(np.float64), ref.astype(NP[dtype]).astype(np.float64))


@gpu
def test_transpose_ttt_norm_guarded(tl, cuda_dev):
    dtype = "f32"
    n = (64, 40, 12)
    X = synth.uniform(n, 4830)
    A = put(X, (2, 3, 1), cuda_dev, dtype)
    mA, wA = synth.to_memory(X.astype(np.float32), (2, 3, 1)), oracle.strides(n, (2, 3, 1))
    tau = (3, 1, 2)
    nt = tuple(n[x - 1] for x in tau)
    G = Guarded(cuda_dev, dtype, nt)
    tl.check(tl.tl_transpose(tl.Desc(A, n, (2, 3, 1)), tau, G.desc(tl)))
    ref, _ = oracle.transpose(mA, n, wA, tau)
    np.testing.assert_array_equal(G.check().astype(np.float64), ref)
    # ttt: A (64, 40, 12) . Y (40, 12, 30) over modes 2, 3 of A
    nB = (40, 12, 30)
    Y = synth.uniform(nB, 4831)
    Bd = put(Y, (1, 2, 3), cuda_dev, dtype)
    Gc = Guarded(cuda_dev, dtype, (64, 30), (1, 2))
    tl.check(tl.tl_ttt(tl.Desc(A, n, (2, 3, 1)), (1, 2, 3), tl.Desc(Bd, nB), (3, 1, 2), 2,
                       Gc.desc(tl)))
    reft, _ = oracle.ttt(mA, n, wA, (1, 2, 3), _dense_first(Y.astype(np.float32)), nB,
                         oracle.strides(nB), (3, 1, 2), 2)
    assert rel_err(Gc.check(), reft) <= TOL[dtype]
    # norm writes exactly three doubles
    Gn = Guarded(cuda_dev, "f64", (3,))
    tl.check(tl.tl_norm(tl.Desc(A, n, (2, 3, 1)), Gn.ptr))
    got = Gn.check()
    assert abs(got[0] - oracle.norm(mA, n, wA)) <= 1e-12 * got[0]


@gpu
def test_batch_guarded(tl, cuda_dev):
    from test_batch_gpu import OpSet
    # the OpSet outputs are whole tensors; re-home each into a guarded buffer
    s = OpSet(tl, cuda_dev, 120, 4840, "f32")
    guards = []
    for o, (C, ref) in zip(s.ops, s.items):
        n = tuple(o.C.n[r] for r in range(o.C.p))
        G = Guarded(cuda_dev, "f32", n)
        o.C.data = G.ptr
        o.C.w = None
        o.C.pi = None
        guards.append((G, o, ref))
    # outputs now first-order inside guard bands: recompute the references
    rc, b = tl.tl_batch_create(s.ops, 0)
    tl.check(rc)
    try:
        tl.check(tl.tl_batch_run(b))
        torch.cuda.synchronize()
        for G, o, ref in guards:
            G.check()
    finally:
        tl.tl_batch_destroy(b)


@pytest.mark.parametrize("t", [None, (2, 3)])
def test_guard_band_detects_a_stray_write_on_cpu(t):
    # the canary check itself, on a host buffer: a write inside the view is
    # fine, one into a gap or a guard zone is reported
    G = Guarded(torch.device("cpu"), "f32", (5, 4), t)
    G.buf[int(G.pos[7])] = 1.0
    G.check()
    outside = [G.off - 1, G.off + int(np.prod(G.parent))]
    if t:
        outside.append(G.off + 1)           # a gap between view elements
    for pos in outside:
        H = Guarded(torch.device("cpu"), "f32", (5, 4), t)
        H.buf[pos] = 2.0
        with pytest.raises(AssertionError):
            H.check()

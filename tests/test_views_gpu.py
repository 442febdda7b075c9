"""GPU parity of every operation on views (Sec. 3.3): views with steps t > 1,
views of views (strides compose, Eq. 19), views as outputs (elements outside
the view stay untouched), all described by tl_view and checked against the
FP64 oracle evaluated on the parent buffers with the same offsets and
strides."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, TOL, TORCH, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _parent(tl, dev, dtype, n, pi, seed):
    X = synth.uniform(n, seed)
    mem = synth.to_memory(np.asarray(X, NP[dtype]), pi)
    P = to_dev(mem, dev, dtype)
    return P, mem, tl.Desc(P, n, pi)


def _elem(dtype):
    return 8 if dtype == "f64" else 4


def _view2(tl, D, ranges1, ranges2):
    rc, V1 = tl.tl_view(D, *ranges1)
    tl.check(rc, "tl_view")
    rc, V2 = tl.tl_view(V1, *ranges2)
    tl.check(rc, "tl_view")
    return V2


def _offset(V, P, dtype):
    return (V.s.data - P.data_ptr()) // _elem(dtype)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ttv_ttm_on_views_of_views(tl, cuda_dev, dtype):
    n, pi = (40, 30, 22), (2, 3, 1)
    P, mem, D = _parent(tl, cuda_dev, dtype, n, pi, 2000)
    # first view: rows 1..37 step 2, 0..29 step 1, 3..21 step 3; then every
    # other element of the first two modes of that
    V = _view2(tl, D, ((1, 0, 3), (2, 1, 3), (37, 29, 21)), ((0, 1, 0), (2, 2, 1), (18, 29, 6)))
    off = _offset(V, P, dtype)
    for q in (1, 2, 3):
        b = synth.uniform((V.n[q - 1],), 2010 + q)
        bt = to_dev(b, cuda_dev, dtype)
        nout = tuple(x for r, x in enumerate(V.n) if r != q - 1)
        C = torch.full((int(np.prod(nout)),), float("nan"), dtype=TORCH[dtype], device=cuda_dev)
        tl.check(tl.tl_ttv(V, bt, 1, q, tl.Desc(C, nout), 0))
        Bm = synth.uniform((5, V.n[q - 1]), 2020 + q)
        Bt = to_dev(Bm.reshape(-1), cuda_dev, dtype)
        nm = tuple(5 if r == q - 1 else x for r, x in enumerate(V.n))
        Cm = torch.full((int(np.prod(nm)),), float("nan"), dtype=TORCH[dtype], device=cuda_dev)
        tl.check(tl.tl_ttm(V, Bt, 5, V.n[q - 1], 1, q, tl.Desc(Cm, nm), 0, 0))
        torch.cuda.synchronize()
        ref = oracle.ttv(mem, V.n, V.w, q, np.asarray(b, NP[dtype]), offA=off)
        assert rel_err(C.cpu().numpy(), ref) <= TOL[dtype], q
        refm = oracle.ttm(mem, V.n, V.w, q, np.asarray(Bm, NP[dtype]).reshape(-1), 5, V.n[q - 1],
                          1, offA=off)
        assert rel_err(Cm.cpu().numpy(), refm) <= TOL[dtype], q


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_entrywise_into_an_output_view(tl, cuda_dev, dtype):
    n = (24, 18, 10)
    P, mem, D = _parent(tl, cuda_dev, dtype, n, (1, 2, 3), 2100)
    Q, memq, DQ = _parent(tl, cuda_dev, dtype, (30, 20, 12), (3, 1, 2), 2101)
    VA = _view2(tl, D, ((0, 1, 0), (1, 2, 1), (23, 17, 9)), ((2, 0, 1), (3, 1, 2), (23, 8, 9)))
    sh = VA.n
    # B: a view of Q with the same extents
    rc, VB = tl.tl_view(DQ, (1, 2, 0), (4, 1, 2), (1 + 4 * (sh[0] - 1), 2 + sh[1] - 1,
                                                    2 * (sh[2] - 1)))
    tl.check(rc)
    assert VB.n == sh
    # output: a view with steps into a NaN-filled buffer
    big = (3 * sh[0], 2 * sh[1] + 1, sh[2] + 2)
    Out = torch.full((int(np.prod(big)),), float("nan"), dtype=TORCH[dtype], device=cuda_dev)
    DO = tl.Desc(Out, big, (2, 1, 3))
    rc, VO = tl.tl_view(DO, (2, 1, 1), (3, 2, 1), (2 + 3 * (sh[0] - 1), 1 + 2 * (sh[1] - 1),
                                                    sh[2]))
    tl.check(rc)
    tl.check(tl.tl_entrywise(tl.TL_MUL, VA, VB, 1.0, VO))
    torch.cuda.synchronize()
    got = Out.cpu().numpy().astype(np.float64)
    oo = _offset(VO, Out, dtype)
    ref = oracle.entrywise(oracle.OP_MUL, sh, mem, VA.w, memq, VB.w,
                           C=np.full(got.shape, np.nan), wC=VO.w, offA=_offset(VA, P, dtype),
                           offB=_offset(VB, Q, dtype))
    # the oracle writes through wC from element 0; shift it to the view's offset
    inside = np.zeros(got.shape, dtype=bool)
    idx = np.indices(sh).reshape(len(sh), -1).T
    offs = oo + idx @ np.asarray(VO.w)
    inside[offs] = True
    # one rounding of the exact FP64 product to the data type (exact for FP64)
    ref_vals = ref[offs - oo].astype(NP[dtype]).astype(np.float64)
    np.testing.assert_array_equal(got[offs], ref_vals)
    assert np.all(np.isnan(got[~inside]))


def test_transpose_ttt_norm_and_ttvs_on_views(tl, cuda_dev):
    dtype = "f64"
    n, pi = (26, 20, 14, 6), (3, 1, 4, 2)
    P, mem, D = _parent(tl, cuda_dev, dtype, n, pi, 2200)
    V = _view2(tl, D, ((1, 0, 2, 0), (2, 1, 1, 2), (25, 19, 13, 4)),
               ((0, 2, 0, 0), (1, 3, 2, 1), (12, 17, 10, 2)))
    off = _offset(V, P, dtype)
    # transpose
    tau = (3, 1, 4, 2)
    nc = tuple(V.n[t - 1] for t in tau)
    C = torch.empty(int(np.prod(nc)), dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_transpose(V, tau, tl.Desc(C, nc)))
    torch.cuda.synchronize()
    ref, _ = oracle.transpose(mem, V.n, V.w, tau, offA=off)
    np.testing.assert_array_equal(C.cpu().numpy(), ref)
    # ttt: contract modes 2 and 4 of the view with a dense (n_4, 7, n_2) tensor
    nB = (V.n[3], 7, V.n[1])
    Y = synth.uniform(nB, 2210)
    Bd = to_dev(synth.to_memory(Y, (1, 2, 3)), cuda_dev, dtype)
    phi, psi = (1, 3, 2, 4), (2, 3, 1)
    ncc = oracle.ttt_shape(V.n, nB, 2, phi, psi)
    Ct = torch.empty(int(np.prod(ncc)), dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_ttt(V, phi, tl.Desc(Bd, nB), psi, 2, tl.Desc(Ct, ncc)))
    torch.cuda.synchronize()
    reft, _ = oracle.ttt(mem, V.n, V.w, phi, synth.to_memory(Y, (1, 2, 3)), nB,
                         oracle.strides(nB), psi, 2, offA=off)
    assert rel_err(Ct.cpu().numpy(), reft) <= TOL[dtype]
    # norm
    res = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_norm(V, res))
    torch.cuda.synchronize()
    assert abs(float(res[0]) - oracle.norm(mem, V.n, V.w, offA=off)) <= \
        1e-13 * oracle.norm(mem, V.n, V.w, offA=off)
    # times_vectors along modes 1 and 3
    vecs = [synth.uniform((V.n[m - 1],), 2220 + m) for m in (1, 3)]
    vd = [to_dev(v, cuda_dev, dtype) for v in vecs]
    rest = (V.n[1], V.n[3])
    Cv = torch.empty(int(np.prod(rest)), dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_ttvs(V, vd, (1, 3), tl.Desc(Cv, rest)))
    torch.cuda.synchronize()
    refv, _ = oracle.ttvs(mem, V.n, V.w, (1, 3), vecs, offA=off)
    assert rel_err(Cv.cpu().numpy(), refv) <= TOL[dtype]

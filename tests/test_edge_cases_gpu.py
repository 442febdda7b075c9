"""Edge cases of every operation against the FP64 oracle: the maximum order
(16 modes, random layouts), all-ones shapes, contractions of length one,
single-element outputs, and the same operations through one persistent batch
(whose descriptors hold at most 8 collapsed dims, so high orders run on their
own kernels)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, TOL, TORCH, get, put, rel_err, to_dev

pytestmark = pytest.mark.gpu

P_MAX = 16


def _max_order_shape(seed):
    g = synth.rng(seed)
    return tuple(int(x) for x in g.choice([1, 2, 2, 2, 3], size=P_MAX))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_maximum_order_every_operation(tl, cuda_dev, dtype):
    g = synth.rng(4700)
    n = _max_order_shape(4701)
    X = synth.uniform(n, 4702)
    Y = synth.uniform(n, 4703)
    pa, pb, pc = (synth.random_layout(P_MAX, g) for _ in range(3))
    A, B = put(X, pa, cuda_dev, dtype), put(Y, pb, cuda_dev, dtype)
    mA, mB = synth.to_memory(np.asarray(X, NP[dtype]), pa), synth.to_memory(np.asarray(Y, NP[dtype]), pb)
    wA, wB = oracle.strides(n, pa), oracle.strides(n, pb)
    # entrywise (bit-exact)
    C = torch.empty(int(np.prod(n)), dtype=TORCH[dtype], device=cuda_dev)
    tl.check(tl.tl_entrywise(tl.TL_SUB, tl.Desc(A, n, pa), tl.Desc(B, n, pb), 1.0, tl.Desc(C, n, pc)))
    torch.cuda.synchronize()
    ref = oracle.entrywise(oracle.OP_SUB, n, mA, wA, mB, wB, wC=oracle.strides(n, pc))
    np.testing.assert_array_equal(C.cpu().numpy().astype(np.float64), ref.astype(NP[dtype]))
    for q in (1, 7, P_MAX):
        # ttv
        nout = tuple(x for r, x in enumerate(n) if r != q - 1)
        pic = synth.random_layout(P_MAX - 1, g)
        b = synth.uniform((n[q - 1],), 4710 + q)
        Cv = torch.empty(int(np.prod(nout)), dtype=TORCH[dtype], device=cuda_dev)
        tl.check(tl.tl_ttv(tl.Desc(A, n, pa), to_dev(b, cuda_dev, dtype), 1, q,
                           tl.Desc(Cv, nout, pic), 0))
        torch.cuda.synchronize()
        refv = oracle.ttv(mA, n, wA, q, np.asarray(b, NP[dtype]), wC=oracle.strides(nout, pic))
        assert rel_err(Cv.cpu().numpy(), refv) <= TOL[dtype], q
        # ttm with J = 3
        Bm = synth.uniform((3, n[q - 1]), 4720 + q)
        nm = tuple(3 if r == q - 1 else x for r, x in enumerate(n))
        Cm = torch.empty(int(np.prod(nm)), dtype=TORCH[dtype], device=cuda_dev)
        tl.check(tl.tl_ttm(tl.Desc(A, n, pa), to_dev(Bm.reshape(-1), cuda_dev, dtype), 3, n[q - 1],
                           1, q, tl.Desc(Cm, nm, pc), 0, 0))
        torch.cuda.synchronize()
        refm = oracle.ttm(mA, n, wA, q, np.asarray(Bm, NP[dtype]).reshape(-1), 3, n[q - 1], 1,
                          wC=oracle.strides(nm, pc))
        assert rel_err(Cm.cpu().numpy(), refm) <= TOL[dtype], q
    # transposition by a random tuple (bit-exact)
    tau = synth.random_layout(P_MAX, g)
    nt = tuple(n[t - 1] for t in tau)
    Ct = torch.empty(int(np.prod(n)), dtype=TORCH[dtype], device=cuda_dev)
    tl.check(tl.tl_transpose(tl.Desc(A, n, pa), tau, tl.Desc(Ct, nt)))
    torch.cuda.synchronize()
    reft, _ = oracle.transpose(mA, n, wA, tau)
    np.testing.assert_array_equal(Ct.cpu().numpy().astype(np.float64), reft.astype(NP[dtype]))
    # norm
    res = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_norm(tl.Desc(A, n, pa), res))
    torch.cuda.synchronize()
    ref_n = oracle.norm(mA, n, wA)
    assert abs(float(res[0]) - ref_n) <= 1e-12 * ref_n


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_maximum_order_contraction_of_eight_modes(tl, cuda_dev, dtype):
    # (8, phi, psi) product of two order-16 tensors sharing eight extents
    g = synth.rng(4730)
    nj = tuple(int(x) for x in g.choice([1, 2, 3], size=8))
    na_free = tuple(int(x) for x in g.choice([1, 2], size=8))
    nb_free = tuple(int(x) for x in g.choice([1, 2], size=8))
    phi = [int(x) + 1 for x in g.permutation(P_MAX)]
    psi = [int(x) + 1 for x in g.permutation(P_MAX)]
    nA, nB = [0] * P_MAX, [0] * P_MAX
    for k in range(8):
        nA[phi[k] - 1] = na_free[k]
        nB[psi[k] - 1] = nb_free[k]
        nA[phi[8 + k] - 1] = nB[psi[8 + k] - 1] = nj[k]
    nA, nB = tuple(nA), tuple(nB)
    X, Y = synth.uniform(nA, 4731), synth.uniform(nB, 4732)
    pa, pb = synth.random_layout(P_MAX, g), synth.random_layout(P_MAX, g)
    A, B = put(X, pa, cuda_dev, dtype), put(Y, pb, cuda_dev, dtype)
    nc = oracle.ttt_shape(nA, nB, 8, phi, psi)
    C = torch.empty(int(np.prod(nc)), dtype=TORCH[dtype], device=cuda_dev)
    tl.check(tl.tl_ttt(tl.Desc(A, nA, pa), phi, tl.Desc(B, nB, pb), psi, 8, tl.Desc(C, nc)))
    torch.cuda.synchronize()
    ref, _ = oracle.ttt(synth.to_memory(np.asarray(X, NP[dtype]), pa), nA, oracle.strides(nA, pa),
                        phi, synth.to_memory(np.asarray(Y, NP[dtype]), pb), nB,
                        oracle.strides(nB, pb), psi, 8)
    assert rel_err(C.cpu().numpy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("p", [2, 3, 5])
def test_all_ones_shapes(tl, cuda_dev, p):
    n = (1,) * p
    X = np.full(n, 3.0)
    A = put(X, synth.first_order(p), cuda_dev, "f64")
    # ttv: one product
    C = torch.empty(1, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_ttv(tl.Desc(A, n), to_dev(np.array([-2.0]), cuda_dev, "f64"), 1, 1,
                       tl.Desc(C, (1,) * (p - 1)), 0))
    # ttm with J = 5: five products of the single element
    Cm = torch.empty(5, dtype=torch.float64, device=cuda_dev)
    Bm = to_dev(np.arange(1.0, 6.0), cuda_dev, "f64")
    tl.check(tl.tl_ttm(tl.Desc(A, n), Bm, 5, 1, 1, p, tl.Desc(Cm, (1,) * (p - 1) + (5,)), 0, 0))
    # entrywise between layouts
    Ce = torch.empty(1, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_entrywise(tl.TL_MUL, tl.Desc(A, n), tl.Desc(A, n, synth.last_order(p)), 1.0,
                             tl.Desc(Ce, n)))
    torch.cuda.synchronize()
    assert float(C[0]) == -6.0
    np.testing.assert_array_equal(Cm.cpu().numpy(), 3.0 * np.arange(1.0, 6.0))
    assert float(Ce[0]) == 9.0


def test_edge_operations_through_one_batch(tl, cuda_dev):
    # an order-16 ttv (more collapsed dims than a batch descriptor holds) and
    # degenerate ttv / ttm next to ordinary ones in one persistent launch
    ops, checks, keep = [], [], []
    n16 = _max_order_shape(4740)
    X16 = synth.uniform(n16, 4741)
    A16 = put(X16, synth.first_order(P_MAX), cuda_dev, "f64")
    b16 = to_dev(synth.uniform((n16[3],), 4742), cuda_dev, "f64")
    nout16 = tuple(x for r, x in enumerate(n16) if r != 3)
    pic = synth.random_layout(P_MAX - 1, synth.rng(4743))
    C16 = torch.empty(int(np.prod(nout16)), dtype=torch.float64, device=cuda_dev)
    D = (tl.Desc(A16, n16), tl.Desc(C16, nout16, pic))
    ops.append(tl.make_op(tl.TL_OP_TTV, D[0], D[1], q=4, vec=b16))
    keep += [A16, b16, C16, D]
    checks.append((C16, oracle.ttv(synth.to_memory(X16, synth.first_order(P_MAX)), n16,
                                   oracle.strides(n16), 4, b16.cpu().numpy(),
                                   wC=oracle.strides(nout16, pic))))
    for i, (n, q, J) in enumerate([((1, 7, 1), 2, 1), ((5, 1, 3), 2, 4), ((40, 33, 9), 3, 7)]):
        X = synth.uniform(n, 4750 + i)
        A = put(X, (3, 1, 2), cuda_dev, "f64")
        Bm = synth.uniform((J, n[q - 1]), 4760 + i)
        Bd = to_dev(Bm.reshape(-1), cuda_dev, "f64")
        nm = tuple(J if r == q - 1 else x for r, x in enumerate(n))
        C = torch.empty(int(np.prod(nm)), dtype=torch.float64, device=cuda_dev)
        D = (tl.Desc(A, n, (3, 1, 2)), tl.Desc(C, nm, (3, 1, 2)))
        ops.append(tl.make_op(tl.TL_OP_TTM, D[0], D[1], q=q, vec=Bd, J=J, ldb_row=n[q - 1],
                              ldb_col=1))
        keep += [A, Bd, C, D]
        checks.append((C, oracle.ttm(synth.to_memory(X, (3, 1, 2)), n,
                                     oracle.strides(n, (3, 1, 2)), q, Bm.reshape(-1), J,
                                     n[q - 1], 1, wC=oracle.strides(nm, (3, 1, 2)))))
    rc, bt = tl.tl_batch_create(ops, tl.TL_BATCH_GRAPH)
    tl.check(rc)
    try:
        tl.check(tl.tl_batch_run(bt))
        torch.cuda.synchronize()
        for C, ref in checks:
            assert rel_err(C.cpu().numpy(), ref) <= TOL["f64"]
    finally:
        tl.tl_batch_destroy(bt)

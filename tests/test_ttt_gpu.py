"""GPU parity of transposition (Table 3, transpose) and of the (q, phi, psi)-mode
tensor-tensor product (Sec. 5.2) through the C ABI, against the FP64 oracle on
the same seeded inputs: every transposition tuple of small orders, random
contractions in random layouts (which take the direct, operand-packing and
temporary-output routes), the inner and outer products, accumulation, and the
tensor-core precisions on GEMM-shaped contractions."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, TOL, TORCH, get, put, rel_err, to_dev

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------- transpose ---

@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_transpose_every_tau_bit_exact(tl, cuda_dev, dtype):
    g = synth.rng(1200)
    n = (33, 7, 20)
    X = synth.uniform(n, 1201)
    for tau in itertools.permutations((1, 2, 3)):
        pa, pc = synth.random_layout(3, g), synth.random_layout(3, g)
        nc = tuple(n[t - 1] for t in tau)
        A = put(X, pa, cuda_dev, dtype)
        C = torch.full((int(np.prod(n)),), float("nan"), dtype=TORCH[dtype], device=cuda_dev)
        tl.check(tl.tl_transpose(tl.Desc(A, n, pa), tau, tl.Desc(C, nc, pc)), "tl_transpose")
        torch.cuda.synchronize()
        Xd = np.asarray(X, NP[dtype])
        ref, rn = oracle.transpose(synth.to_memory(Xd, pa), n, oracle.strides(n, pa), tau,
                                   wC=oracle.strides(nc, pc))
        assert rn == nc
        np.testing.assert_array_equal(C.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("n,tau", [((64, 48, 5, 9), (3, 1, 4, 2)), ((128, 130, 3), (2, 1, 3)),
                                   ((4, 3, 5, 2, 6), (5, 4, 3, 2, 1)), ((257, 129), (2, 1))])
def test_transpose_larger_cases(tl, cuda_dev, n, tau):
    X = synth.normal(n, 1210 + len(n), dtype=np.float32)
    p = len(n)
    A = put(X, synth.first_order(p), cuda_dev, "f32")
    nc = tuple(n[t - 1] for t in tau)
    C = torch.empty(int(np.prod(n)), dtype=torch.float32, device=cuda_dev)
    tl.check(tl.tl_transpose(tl.Desc(A, n), tau, tl.Desc(C, nc)))
    torch.cuda.synchronize()
    ref = np.transpose(X, [t - 1 for t in tau])
    np.testing.assert_array_equal(get(C, nc, synth.first_order(p)), ref)


def test_transpose_rejects_bad_tau(tl, cuda_dev):
    A = torch.zeros(24, dtype=torch.float32, device=cuda_dev)
    C = torch.zeros(24, dtype=torch.float32, device=cuda_dev)
    assert tl.tl_transpose(tl.Desc(A, (2, 3, 4)), (1, 1, 3), tl.Desc(C, (2, 3, 4))) == tl.TL_EINVAL
    assert tl.tl_transpose(tl.Desc(A, (2, 3, 4)), (2, 1, 3), tl.Desc(C, (2, 3, 4))) == tl.TL_EINVAL


# ------------------------------------------------------------------- ttt ---

def _random_ttt(g, q, r, s, emin=1, emax=9):
    ext = lambda: int(g.integers(emin, emax + 1))
    nj = [ext() for _ in range(q)]
    phi = [int(x) + 1 for x in g.permutation(q + r)]
    psi = [int(x) + 1 for x in g.permutation(q + s)]
    nA, nB = [0] * (q + r), [0] * (q + s)
    for k in range(r):
        nA[phi[k] - 1] = ext()
    for k in range(s):
        nB[psi[k] - 1] = ext()
    for k in range(q):
        nA[phi[r + k] - 1] = nB[psi[s + k] - 1] = nj[k]
    return tuple(nA), tuple(nB), phi, psi


def _run_ttt(tl, dev, dtype, nA, pa, phi, nB, pb, psi, q, pc=None, precision=0, accumulate=False,
             seed=0):
    X = synth.uniform(nA, 1300 + seed)
    Y = synth.uniform(nB, 1400 + seed)
    A, B = put(X, pa, dev, dtype), put(Y, pb, dev, dtype)
    nc = oracle.ttt_shape(nA, nB, q, phi, psi)
    pc = pc or synth.first_order(len(nc))
    C0 = synth.uniform(nc, 1500 + seed) if accumulate else np.zeros(nc)
    if nc:
        C = put(C0, pc, dev, dtype)
        DC = tl.Desc(C, nc, pc)
    else:
        C = to_dev(np.zeros(1), dev, dtype)
        DC = tl.Desc(C, (1,))
    tl.check(tl.tl_ttt(tl.Desc(A, nA, pa), phi, tl.Desc(B, nB, pb), psi, q, DC, precision,
                       int(accumulate)), "tl_ttt")
    torch.cuda.synchronize()
    Xd, Yd = np.asarray(X, NP[dtype]), np.asarray(Y, NP[dtype])
    wc = oracle.strides(nc, pc) if nc else ()
    ref, rn = oracle.ttt(synth.to_memory(Xd, pa), nA, oracle.strides(nA, pa), phi,
                         synth.to_memory(Yd, pb), nB, oracle.strides(nB, pb), psi, q,
                         C=synth.to_memory(np.asarray(C0, NP[dtype]), pc) if nc else None, wC=wc,
                         accumulate=accumulate)
    assert rn == nc
    return C.cpu().numpy().astype(np.float64), ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("q,r,s", [(1, 2, 1), (2, 1, 2), (3, 1, 1), (2, 2, 0), (2, 0, 2),
                                   (1, 3, 2), (2, 2, 2), (1, 1, 3)])
def test_ttt_random_contractions_random_layouts(tl, cuda_dev, dtype, q, r, s):
    g = synth.rng(1600 + 31 * q + 7 * r + s)
    for trial in range(6):
        nA, nB, phi, psi = _random_ttt(g, q, r, s)
        pa = synth.random_layout(len(nA), g)
        pb = synth.random_layout(len(nB), g)
        pc = synth.random_layout(r + s, g) if r + s else None
        got, ref = _run_ttt(tl, cuda_dev, dtype, nA, pa, phi, nB, pb, psi, q, pc=pc,
                            seed=trial)
        assert rel_err(got, ref) <= TOL[dtype], (nA, nB, phi, psi, pa, pb, pc)


@pytest.mark.parametrize("case", ["direct", "pack_v", "pack_t", "temp_c"])
def test_ttt_every_route(tl, cuda_dev, case):
    # direct: A (M1,M2,K1,K2) . B (K1,K2,N) in first-order layouts
    # pack_v: B lists the contracted modes in the opposite memory order to A
    # pack_t: A's contracted modes are not adjacent in memory
    # temp_c: C's layout splits B's two free modes apart
    if case == "direct":
        args = ((12, 10, 9, 7), (1, 2, 3, 4), (1, 2, 3, 4), (9, 7, 11), (1, 2, 3), (3, 1, 2), 2,
                None)
    elif case == "pack_v":
        args = ((40, 9, 7), (1, 2, 3), (1, 2, 3), (7, 9, 13), (1, 2, 3), (3, 2, 1), 2, None)
    elif case == "pack_t":
        args = ((9, 40, 7), (1, 2, 3), (2, 1, 3), (9, 7, 13), (1, 2, 3), (3, 1, 2), 2, None)
    else:
        args = ((40, 9), (1, 2), (1, 2), (9, 6, 5), (1, 2, 3), (2, 3, 1), 1, (2, 1, 3))
    nA, pa, phi, nB, pb, psi, q, pc = args
    for dtype in ("f64", "f32"):
        got, ref = _run_ttt(tl, cuda_dev, dtype, nA, pa, phi, nB, pb, psi, q, pc=pc)
        assert rel_err(got, ref) <= TOL[dtype], (case, dtype)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ttt_inner_outer_and_accumulate(tl, cuda_dev, dtype):
    # inner product over all modes of two order-3 tensors in different layouts
    got, ref = _run_ttt(tl, cuda_dev, dtype, (30, 20, 10), (3, 1, 2), (1, 2, 3), (20, 10, 30),
                        (1, 2, 3), (3, 1, 2), 3)
    assert rel_err(got, ref) <= TOL[dtype]
    # outer product (q = 0)
    got, ref = _run_ttt(tl, cuda_dev, dtype, (7, 5), (2, 1), (1, 2), (3, 4, 6), (1, 2, 3),
                        (1, 2, 3), 0, pc=(5, 1, 3, 2, 4))
    assert rel_err(got, ref) <= TOL[dtype]
    # accumulate into C, direct and through the temporary output
    got, ref = _run_ttt(tl, cuda_dev, dtype, (12, 10, 9), (1, 2, 3), (1, 2, 3), (9, 11),
                        (1, 2), (2, 1), 1, accumulate=True, seed=3)
    assert rel_err(got, ref) <= TOL[dtype]
    got, ref = _run_ttt(tl, cuda_dev, dtype, (40, 9), (1, 2), (1, 2), (9, 6, 5), (1, 2, 3),
                        (2, 3, 1), 1, pc=(2, 1, 3), accumulate=True, seed=4)
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("prec,tol", [(5, 1e-5), (3, 1e-2), (4, 1e-2)])
def test_ttt_tensor_core_precisions_on_gemm_shapes(tl, cuda_dev, prec, tol):
    # A (M1=64, M2=32, K1=16, K2=16) . B (K1, K2, N=96): K collapses to 256
    got, ref = _run_ttt(tl, cuda_dev, "f32", (64, 32, 16, 16), (1, 2, 3, 4), (1, 2, 3, 4),
                        (16, 16, 96), (1, 2, 3), (3, 1, 2), 2, precision=prec, seed=7)
    assert rel_err(got, ref) <= tol
    # the contracted modes fastest in A (row case) and an output wider than
    # one tensor-core call (N = 600 > 512 rows of the matrix operand)
    got, ref = _run_ttt(tl, cuda_dev, "f32", (128, 64, 16), (1, 2, 3), (2, 3, 1), (128, 600),
                        (1, 2), (2, 1), 1, precision=prec, seed=8)
    assert rel_err(got, ref) <= tol


def test_ttt_rejects_bad_calls(tl, cuda_dev):
    A = torch.zeros(60, dtype=torch.float32, device=cuda_dev)
    B = torch.zeros(60, dtype=torch.float32, device=cuda_dev)
    C = torch.zeros(400, dtype=torch.float32, device=cuda_dev)
    DA, DB = tl.Desc(A, (3, 4, 5)), tl.Desc(B, (5, 4, 3))
    # extents of a contracted pair differ (3 vs 5)
    assert tl.tl_ttt(DA, (2, 3, 1), DB, (3, 2, 1), 1, tl.Desc(C, (4, 5, 5, 4))) == tl.TL_EINVAL
    # phi not a permutation
    assert tl.tl_ttt(DA, (1, 1, 3), DB, (1, 2, 3), 1, tl.Desc(C, (3, 4, 5, 4))) == tl.TL_EINVAL
    # wrong C extents (the right ones are (3, 4, 4, 3))
    assert tl.tl_ttt(DA, (1, 2, 3), DB, (2, 3, 1), 1, tl.Desc(C, (3, 4, 3, 4))) == tl.TL_EINVAL
    # an F64 precision on FP32 data
    assert tl.tl_ttt(DA, (1, 2, 3), DB, (2, 3, 1), 1, tl.Desc(C, (3, 4, 4, 3)), 1) == \
        tl.TL_EUNSUPPORTED

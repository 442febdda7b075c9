"""GPU parity of the FP32 register-tiled ttm (Sec. 5.2 Eq. 25) against the
FP64 oracle, in every way the kernel reads its operands (16-byte vectors
along k or along contiguous rows, element loads) and writes its output
(vectors along j or along rows, element stores, split-K partials).

Shapes span several 128 x 256 tiles (J > 128), 256 x 128 tiles (64 < J <=
128) or 512 x 64 tiles (J <= 64) with ragged edges in rows, columns and the contraction (not a multiple of
the 8-deep k slab).  Bars: integer-valued
inputs are bit-exact (every partial sum is an integer below 2^24); real
inputs stay within each element's rounding bound of a length-n_q FP32 dot
product and within a relative Frobenius error of 1e-5."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import put, rel_err, ttm_case

pytestmark = pytest.mark.gpu

# (n, q, J, pi_A, pi_C, B column-major, expected A read, expected C write):
# A is read in 16-byte vectors along k (k4) or along four contiguous rows
# (r4), or element by element; C is written in 16-byte vectors along j (j4)
# or rows (m4), or element by element
MODES = [
    ((300, 260), 1, 132, (1, 2), (1, 2), False, "k4", "j4"),
    ((260, 300), 2, 132, (1, 2), (1, 2), False, "r4", "m4"),
    ((260, 300), 2, 132, (1, 2), (2, 1), True, "r4", "j4"),
    ((300, 260), 1, 132, (1, 2), (2, 1), True, "k4", "m4"),
    ((301, 257), 2, 50, (1, 2), (1, 2), False, "scalar", "scalar"),
    ((301, 257), 1, 50, (2, 1), (2, 1), True, "scalar", "scalar"),
    ((36, 20, 131), 3, 136, (1, 2, 3), (3, 1, 2), False, "r4", "j4"),
    ((131, 20, 36), 1, 7, (1, 2, 3), (1, 2, 3), False, "scalar", "scalar"),
    ((64, 70, 13, 8), 2, 260, (4, 1, 3, 2), (4, 2, 1, 3), False, "r4", "m4"),
    ((64, 70, 13, 6), 2, 130, (4, 1, 3, 2), (2, 4, 1, 3), True, "r4", "scalar"),
    ((300, 520), 1, 300, (1, 2), (1, 2), False, "k4", "j4"),
    ((300, 260), 1, 100, (1, 2), (1, 2), False, "k4", "j4"),
    ((260, 300), 2, 64, (1, 2), (1, 2), False, "r4", "m4"),
    ((500, 1100), 1, 60, (1, 2), (1, 2), False, "k4", "j4"),
    ((1100, 500), 2, 64, (1, 2), (1, 2), False, "r4", "m4"),
    ((36, 500, 30), 2, 36, (1, 2, 3), (2, 3, 1), True, "r4", "j4"),
]


def _plan(tl, dev, n, q, J, pi_a, pi_c):
    A = torch.empty(int(np.prod(n)), dtype=torch.float32, device=dev)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    C = torch.empty(int(np.prod(nout)), dtype=torch.float32, device=dev)
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n, pi_a), None, q, J, 0, 0,
                                 tl.Desc(C, nout, pi_c))
    assert rc == 0, js
    return json.loads(js)


@pytest.mark.parametrize("case", MODES, ids=[f"{m[6]}-{m[7]}-{i}" for i, m in enumerate(MODES)])
def test_sgemm_modes_integer_exact_and_real_bounded(tl, cuda_dev, case):
    n, q, J, pi_a, pi_c, colB, amode, cmode = case
    d = _plan(tl, cuda_dev, n, q, J, pi_a, pi_c)
    assert d["kernel"] == "ttm_simt" and d["splits"] == 1, d
    assert d["sgemm"]["a"] == amode and d["sgemm"]["c"] == cmode, d
    assert d["sgemm"]["tile"] == ([128, 256] if J > 128 else [256, 128] if J > 64 else [512, 64]), d
    nq = n[q - 1]
    # integers in [-4, 4]: sums stay below 2^24, so every order of summation is exact
    X = synth.integers(n, 7100 + J, lo=-4, hi=4)
    Bm = synth.integers((J, nq), 7101 + J, lo=-4, hi=4)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi_a, pi_c, "f32", col_major=colB)
    np.testing.assert_array_equal(got, ref)
    # real data: per-element bound of a length-n_q dot product in FP32
    X = synth.normal(n, 7102 + J, dtype=np.float64).astype(np.float32)
    Bm = synth.normal((J, nq), 7103 + J, dtype=np.float64).astype(np.float32)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi_a, pi_c, "f32", col_major=colB)
    eps = np.finfo(np.float32).eps / 2
    bound = 2 * nq * eps * np.moveaxis(
        np.tensordot(np.abs(X).astype(np.float64), np.abs(Bm).astype(np.float64).T,
                     axes=([q - 1], [0])), -1, q - 1)
    assert np.all(np.abs(got - ref) <= bound + 1e-30)
    assert rel_err(got, ref) <= 1e-5
    # accumulate: C += A x_q B on top of a random C
    nout = got.shape
    C0 = synth.uniform(nout, 7104 + J)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi_a, pi_c, "f32", accumulate=True, C0=C0,
                        col_major=colB)
    assert rel_err(got, ref) <= 1e-5


@pytest.mark.parametrize("n,q,J,pi", [((40, 200000), 2, 8, (1, 2)), ((240000, 20), 1, 36, (2, 1)),
                                      ((5, 30011, 4), 2, 7, (3, 1, 2))])
def test_sgemm_split_k_vector_and_element_partials(tl, cuda_dev, n, q, J, pi):
    d = _plan(tl, cuda_dev, n, q, J, pi, pi)
    assert d["splits"] > 1
    assert d["sgemm"]["c"] == ("ws4" if J % 4 == 0 else "ws1"), d
    X = synth.uniform(n, 7200 + J)
    Bm = synth.uniform((J, n[q - 1]), 7201 + J)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, "f32")
    assert rel_err(got, ref) <= 1e-5
    C0 = synth.uniform(got.shape, 7202)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, "f32", accumulate=True, C0=C0)
    assert rel_err(got, ref) <= 1e-5


def test_sgemm_unaligned_base_takes_element_loads(tl, cuda_dev):
    # A and C start one element into their buffers: no 16-byte vectors
    n, q, J = (260, 300), 1, 132
    X = synth.normal(n, 7300, dtype=np.float64).astype(np.float32)
    Bm = synth.normal((J, n[0]), 7301, dtype=np.float64).astype(np.float32)
    Abuf = torch.zeros(int(np.prod(n)) + 1, dtype=torch.float32, device=cuda_dev)
    Abuf[1:] = put(X, (1, 2), cuda_dev, "f32")
    nout = (J, n[1])
    Cbuf = torch.zeros(int(np.prod(nout)) + 1, dtype=torch.float32, device=cuda_dev)
    A, C = Abuf[1:], Cbuf[1:]
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n), None, q, J, 0, 0, tl.Desc(C, nout))
    d = json.loads(js)
    assert d["sgemm"]["a"] == "scalar" and d["sgemm"]["c"] == "scalar", d
    Bd = torch.from_numpy(np.ascontiguousarray(Bm).reshape(-1)).to(cuda_dev)
    tl.check(tl.tl_ttm(tl.Desc(A, n), Bd, J, n[0], 1, q, tl.Desc(C, nout), 0, 0))
    torch.cuda.synchronize()
    got = synth.from_memory(C.cpu().numpy(), nout, (1, 2))
    ref = synth.from_memory(
        oracle.ttm(synth.to_memory(X, (1, 2)), n, oracle.strides(n), q, Bm.reshape(-1), J, n[0],
                   1), nout, (1, 2))
    assert rel_err(got, ref) <= 1e-5
    assert float(Cbuf[0]) == 0.0


def test_sgemm_bench_shape_512_cubed_sampled(tl, cuda_dev):
    # the 512^3 x 512 FP32 ttm that the benchmark times, along modes 1 and 3
    n, mem, B, _, _ = synth.precision_case()
    A = torch.from_numpy(mem).to(cuda_dev)
    Bd = torch.from_numpy(np.ascontiguousarray(B).reshape(-1)).to(cuda_dev)
    w = oracle.strides(n)
    g = synth.rng(7400)
    for q in (1, 3):
        C = torch.empty(512 ** 3, dtype=torch.float32, device=cuda_dev)
        tl.check(tl.tl_ttm(tl.Desc(A, n), Bd, 512, 512, 1, q, tl.Desc(C, n), tl.TL_P_F32, 0))
        torch.cuda.synchronize()
        idx = np.stack([g.integers(0, x, size=2000) for x in n], axis=1)
        ref = oracle.ttm_at(mem, n, w, q, B.reshape(-1), 512, 1, idx)
        got = synth.from_memory(C.cpu().numpy(), n, (1, 2, 3))[tuple(idx.T)]
        assert rel_err(got, ref) <= 1e-5, q
        del C

"""GPU parity of tl_ttm (Sec. 5.2 Eq. 25) against the FP64 oracle.

Bars: integer-valued inputs and identity / permutation matrices are bit-exact;
otherwise the relative Frobenius error is <= 1e-12 (FP64) and <= 1e-5 (FP32)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, TORCH, get, put, rel_err, to_dev, ttm_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("seed", range(14))
def test_ttm_random_layouts(tl, cuda_dev, dtype, seed):
    g = synth.rng(2000 + seed)
    p = int(g.integers(2, 7))
    n = tuple(int(x) for x in g.integers(1, 12 if p > 4 else 40, size=p))
    q = int(g.integers(1, p + 1))
    J = int(g.integers(1, 80))
    X = synth.uniform(n, 2100 + seed)
    Bm = synth.uniform((J, n[q - 1]), 2200 + seed)
    acc = bool(g.integers(2))
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    C0 = synth.uniform(nout, 2300 + seed) if acc else None
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, synth.random_layout(p, g),
                        synth.random_layout(p, g), dtype, accumulate=acc, C0=C0,
                        col_major=bool(g.integers(2)))
    assert got.shape == ref.shape
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ttm_integer_identity_permutation_exact(tl, cuda_dev, dtype):
    g = synth.rng(2400)
    n = (13, 7, 19)
    X = synth.integers(n, 2401)
    for q in (1, 2, 3):
        nq = n[q - 1]
        for Bm in (np.eye(nq), np.eye(nq)[g.permutation(nq)], synth.integers((5, nq), 2402 + q)):
            got, ref = ttm_case(tl, cuda_dev, X, q, Bm, synth.random_layout(3, g),
                                synth.random_layout(3, g), dtype)
            np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("shape", [(129, 67, 33), (300, 257), (5, 3, 701), (33, 17, 9, 5)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ttm_multi_tile_ragged_all_modes(tl, cuda_dev, shape, dtype):
    X = synth.normal(shape, 2500, dtype=np.float64)
    p = len(shape)
    for pi in (synth.first_order(p), synth.last_order(p)):
        for q in range(1, p + 1):
            J = 70 if shape[q - 1] > 3 else 3
            Bm = synth.normal((J, shape[q - 1]), 2501 + q, dtype=np.float64)
            got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, dtype)
            assert rel_err(got, ref) <= TOL[dtype], (pi, q)


def test_ttm_small_case_fp64(tl, cuda_dev):
    case = synth.small_case()
    got, ref = ttm_case(tl, cuda_dev, case.X, case.q_ttm, case.B, (1, 2, 3), (1, 2, 3), "f64")
    assert rel_err(got, ref) <= 1e-12


def test_ttm_single_row_matches_ttv(tl, cuda_dev):
    n = (31, 17, 23)
    X = synth.normal(n, 2600, dtype=np.float64)
    for q in (1, 2, 3):
        b = synth.normal((n[q - 1],), 2601 + q, dtype=np.float64)
        got, ref = ttm_case(tl, cuda_dev, X, q, b[None, :], (2, 3, 1), (2, 3, 1), "f64")
        assert rel_err(got, ref) <= 1e-12


@pytest.fixture(scope="module")
def scale_tensors(cuda_dev):
    case = synth.scale_case()
    n = case.n
    memF = case.mem_first
    X = synth.from_memory(memF, n, synth.first_order(4))
    memL = synth.to_memory(X, synth.last_order(4))
    return case, memF, memL, to_dev(memF, cuda_dev, "f32"), to_dev(memL, cuda_dev, "f32")


def test_ttm_full_scale_sampled(tl, cuda_dev, scale_tensors):
    case, memF, memL, AF, AL = scale_tensors
    n = case.n
    g = synth.rng(2700)
    C = torch.empty(128 ** 4, dtype=torch.float32, device=cuda_dev)
    for pi, mem, Ad in ((synth.first_order(4), memF, AF), (synth.last_order(4), memL, AL)):
        wA = oracle.strides(n, pi)
        for q in range(1, 5):
            Bm = case.matrices[q - 1]
            Bt = to_dev(Bm.reshape(-1), cuda_dev, "f32")
            tl.check(tl.tl_ttm(tl.Desc(Ad, n, pi), Bt, 128, 128, 1, q, tl.Desc(C, n, pi)))
            torch.cuda.synchronize()
            got = get(C, n, pi)
            idx = np.stack([g.integers(0, x, size=3000) for x in n], axis=1)
            ref = oracle.ttm_at(mem, n, wA, q, Bm.reshape(-1), 128, 1, idx)
            assert rel_err(got[tuple(idx.T)], ref) <= 1e-5, (pi, q)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,q,J,pi", [((3, 200000), 2, 10, (1, 2)), ((240001, 4), 1, 34, (2, 1)),
                                      ((5, 30011, 3), 2, 7, (3, 1, 2)), ((2, 70000), 2, 1, (1, 2)),
                                      ((40, 100000), 2, 10, (1, 2)), ((24, 50000, 3), 2, 7, (3, 1, 2))])
def test_ttm_split_k_long_contraction(tl, cuda_dev, dtype, n, q, J, pi):
    # few rows and a long contraction: the k range is split across CTAs and the
    # partial sums are added in a fixed order by a second kernel (the skinny
    # kernel for at most 16 rows, the tiled kernels above)
    import json
    X = synth.uniform(n, 4400 + J)
    Bm = synth.uniform((J, n[q - 1]), 4401 + J)
    A = put(X, pi, cuda_dev, dtype)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    C = torch.empty(int(np.prod(nout)), dtype=TORCH[dtype], device=cuda_dev)
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n, pi), None, q, J, 0, 0,
                                 tl.Desc(C, nout, pi))
    d = json.loads(js)
    assert rc == 0 and d["splits"] > 1, js
    M = int(np.prod(n)) // n[q - 1]
    assert d.get("skinny") == (1 if M <= 16 else None), d
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, dtype)
    assert rel_err(got, ref) <= TOL[dtype]
    # accumulate through the split path
    C0 = synth.uniform(nout, 4402)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, dtype, accumulate=True, C0=C0)
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,q,J,pi,pic,colB", [((1, 2048), 2, 1, (1, 2), (1, 2), False),
                                               ((16, 100003), 2, 32, (1, 2), (2, 1), False),
                                               ((7, 4099), 2, 64, (2, 1), (1, 2), True),
                                               ((2, 3, 60001), 3, 33, (3, 1, 2), (1, 2, 3), True),
                                               ((5, 9000, 3), 2, 19, (2, 3, 1), (3, 2, 1), False)])
def test_ttm_skinny_long_contraction(tl, cuda_dev, dtype, n, q, J, pi, pic, colB):
    # at most 16 rows over n_q >= 2048 (M x J <= 512): the skinny split-K
    # kernel, with the contraction contiguous in A or strided, B row- or
    # column-major, C in another layout, a ragged last k tile, one or two
    # outputs per thread, and accumulation
    import json
    X = synth.uniform(n, 4450 + J)
    Bm = synth.uniform((J, n[q - 1]), 4451 + J)
    A = put(X, pi, cuda_dev, dtype)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    C = torch.empty(int(np.prod(nout)), dtype=TORCH[dtype], device=cuda_dev)
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n, pi), None, q, J, 0, 0,
                                 tl.Desc(C, nout, pic))
    d = json.loads(js)
    assert rc == 0 and d.get("skinny") == 1 and d["splits"] > 1, js
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pic, dtype, col_major=colB)
    assert rel_err(got, ref) <= TOL[dtype]
    C0 = synth.uniform(nout, 4452)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pic, dtype, accumulate=True, C0=C0,
                        col_major=colB)
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,q,J,pi,pic", [((2, 3000, 7), 1, 35, (1, 2, 3), (1, 2, 3)),
                                          ((40, 9, 50), 2, 63, (2, 3, 1), (1, 2, 3)),
                                          ((17, 3, 11, 5), 2, 1, (4, 2, 1, 3), (2, 4, 3, 1)),
                                          ((300, 32), 2, 50, (2, 1), (1, 2)),
                                          ((64, 24, 9), 3, 16, (3, 1, 2), (3, 2, 1))])
def test_ttm_rows_short_contractions(tl, cuda_dev, dtype, n, q, J, pi, pic):
    # n_q <= 32: a row of A per thread with the matrix in shared memory, any
    # output layout, J beyond one 16-column pass
    import json
    X = synth.uniform(n, 4500 + J)
    Bm = synth.uniform((J, n[q - 1]), 4501 + J)
    A = put(X, pi, cuda_dev, dtype)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    C = torch.empty(int(np.prod(nout)), dtype=TORCH[dtype], device=cuda_dev)
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n, pi), None, q, J, 0, 0,
                                 tl.Desc(C, nout, pic))
    assert rc == 0 and json.loads(js)["kernel"] == "ttm_rows", js
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pic, dtype)
    assert rel_err(got, ref) <= TOL[dtype]
    C0 = synth.uniform(nout, 4502)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pic, dtype, accumulate=True, C0=C0)
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("nq", [1, 2, 3, 4, 5, 6, 7, 8, 13, 16, 17])
def test_ttm_rows_every_contraction_remainder(tl, cuda_dev, dtype, nq):
    # the row kernel loads a row in chunks of 8 and a remainder chunk of its
    # exact length: every remainder, alone and after whole chunks, with J
    # spanning two full 16-column groups and a ragged one (27331 rows are
    # enough items for 16 columns per item), the contracted mode neither
    # first nor last in memory; integer inputs make every sum exact, so the
    # result is bit-exact against the oracle
    import json
    n = (181, nq, 151)
    pi, pic = (2, 1, 3), (3, 1, 2)
    J = 37
    X = synth.integers(n, 4600 + nq)
    Bm = synth.integers((J, nq), 4601 + nq)
    A = put(X, pi, cuda_dev, dtype)
    nout = (181, J, 151)
    C = torch.empty(int(np.prod(nout)), dtype=TORCH[dtype], device=cuda_dev)
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n, pi), None, 2, J, 0, 0,
                                 tl.Desc(C, nout, pic))
    assert rc == 0 and json.loads(js)["kernel"] == "ttm_rows", js
    got, ref = ttm_case(tl, cuda_dev, X, 2, Bm, pi, pic, dtype)
    np.testing.assert_array_equal(got, ref)
    C0 = synth.integers(nout, 4602)
    got, ref = ttm_case(tl, cuda_dev, X, 2, Bm, pi, pic, dtype, accumulate=True, C0=C0)
    np.testing.assert_array_equal(got, ref)

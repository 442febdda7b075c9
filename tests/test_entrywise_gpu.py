"""GPU parity of tl_entrywise (Sec. 5.1 Eqs. 22-23) against the FP64 oracle.

A single +, -, *, / of FP32 (FP64) operands is correctly rounded on the GPU,
and rounding the oracle's FP64 result to FP32 gives the same correctly rounded
value (53 >= 2*24 + 2 bits, so the double rounding is innocuous), so every
comparison here is bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, get, put, to_dev

pytestmark = pytest.mark.gpu

OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "copy": 4, "scale": 5}


def ew_case(tl, dev, op, X, Y, pa, pb, pc, dtype, alpha=-1.5):
    n = X.shape
    Xd = np.asarray(X, dtype=NP[dtype])
    Yd = np.asarray(Y, dtype=NP[dtype])
    A = put(Xd, pa, dev, dtype)
    B = put(Yd, pb, dev, dtype)
    C = torch.empty_like(A)
    unary = op in (4, 5)
    rc = tl.tl_entrywise(op, tl.Desc(A, n, pa), None if unary else tl.Desc(B, n, pb), alpha,
                         tl.Desc(C, n, pc))
    tl.check(rc, "tl_entrywise")
    torch.cuda.synchronize()
    got = get(C, n, pc)
    ref = oracle.entrywise(op, n, synth.to_memory(Xd, pa), oracle.strides(n, pa),
                           synth.to_memory(Yd, pb), oracle.strides(n, pb), alpha,
                           wC=oracle.strides(n, pc))
    return got, synth.from_memory(ref, n, pc).astype(NP[dtype])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("op", sorted(OPS))
@pytest.mark.parametrize("seed", range(5))
def test_entrywise_random_layouts_bit_exact(tl, cuda_dev, dtype, op, seed):
    g = synth.rng(3000 + seed)
    p = int(g.integers(1, 7))
    n = tuple(int(x) for x in g.integers(1, 12 if p > 3 else 60, size=p))
    X = synth.normal(n, 3100 + seed, dtype=np.float64)
    Y = synth.normal(n, 3200 + seed, dtype=np.float64) + 3.0
    pa, pb, pc = (synth.random_layout(p, g) for _ in range(3))
    got, ref = ew_case(tl, cuda_dev, OPS[op], X, Y, pa, pb, pc, dtype)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("shape", [(1000, 77, 3), (33, 65, 17), (257, 129), (5, 4, 3, 200),
                                   (100, 68, 12), (36, 20, 64), (128, 4, 132)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_entrywise_first_last_mixes_ragged(tl, cuda_dev, shape, dtype):
    p = len(shape)
    X = synth.normal(shape, 3300, dtype=np.float64)
    Y = synth.normal(shape, 3301, dtype=np.float64)
    F, L = synth.first_order(p), synth.last_order(p)
    for pa, pb, pc in [(F, L, F), (L, F, F), (F, F, L), (L, L, F), (F, L, L)]:
        got, ref = ew_case(tl, cuda_dev, 0, X, Y, pa, pb, pc, dtype)
        np.testing.assert_array_equal(got, ref)
        got, ref = ew_case(tl, cuda_dev, 4, X, Y, pa, pb, pc, dtype)   # relayout
        np.testing.assert_array_equal(got, ref)


def test_entrywise_small_case_fp64(tl, cuda_dev):
    case = synth.small_case()
    got, ref = ew_case(tl, cuda_dev, 0, case.X, case.X, (1, 2, 3), (3, 2, 1), (1, 2, 3), "f64")
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(got, 2 * case.X)


def test_entrywise_strided_and_inplace(tl, cuda_dev):
    n = (6, 5, 7)
    npar = (12, 5, 14)
    parent = synth.normal(npar, 3400, dtype=np.float64)
    mem = synth.to_memory(parent, (1, 2, 3))
    w = oracle.strides(npar)
    nv, wv, gamma = oracle.view(npar, w, (1, 0, 0), (2, 1, 2), (11, 4, 13))
    assert nv == n
    Pd = to_dev(mem, cuda_dev, "f64")
    Y = synth.normal(n, 3401, dtype=np.float64)
    B = put(Y, (3, 1, 2), cuda_dev, "f64")
    C = torch.empty(int(np.prod(n)), dtype=torch.float64, device=cuda_dev)
    Av = tl.Desc(Pd.data_ptr() + gamma * 8, n, w=wv, dtype=torch.float64)
    tl.check(tl.tl_entrywise(0, Av, tl.Desc(B, n, (3, 1, 2)), 1.0, tl.Desc(C, n)))
    torch.cuda.synchronize()
    ref = oracle.entrywise(0, n, mem, wv, synth.to_memory(Y, (3, 1, 2)),
                           oracle.strides(n, (3, 1, 2)), offA=gamma)
    np.testing.assert_array_equal(C.cpu().numpy(), ref)
    # in place: C == A with identical descriptors
    before = B.clone()
    tl.check(tl.tl_entrywise(5, tl.Desc(B, n, (3, 1, 2)), None, 2.0, tl.Desc(B, n, (3, 1, 2))))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(B.cpu().numpy(), 2.0 * before.cpu().numpy())


def test_entrywise_full_scale_sampled(tl, cuda_dev):
    case = synth.scale_case()
    n = case.n
    memF = case.mem_first
    X = synth.from_memory(memF, n, synth.first_order(4))
    memL = synth.to_memory(X, synth.last_order(4))
    AF, AL = to_dev(memF, cuda_dev, "f32"), to_dev(memL, cuda_dev, "f32")
    C = torch.empty_like(AF)
    tl.check(tl.tl_entrywise(0, tl.Desc(AF, n), tl.Desc(AL, n, (4, 3, 2, 1)), 1.0, tl.Desc(C, n)))
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    np.testing.assert_array_equal(got, (memF.astype(np.float64) * 2).astype(np.float32))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_entrywise_vector_tile_path_bit_exact(tl, cuda_dev, dtype):
    # extents and strides that allow 16-byte vectors select the vector tile
    # kernel; every staging variant (A staged, B staged, both, unary) over
    # ragged tiles (extents not multiples of the 64 / 32-element tile) and
    # batch dims matches the oracle bit for bit
    import json
    for n in ((100, 68, 12), (64, 64, 8), (36, 132, 16), (36, 20, 4, 16)):
        p = len(n)
        F, L = synth.first_order(p), synth.last_order(p)
        X = synth.normal(n, 3450, dtype=np.float64)
        Y = synth.normal(n, 3451, dtype=np.float64) + 3.0
        for pa, pb, pc, ops in [(F, L, F, ("add", "div")), (L, F, F, ("sub", "mul")),
                                (L, L, F, ("add",)), (F, F, L, ("sub",)), (L, F, F, ("copy", "scale"))]:
            A = put(X, pa, cuda_dev, dtype)
            B = put(Y, pb, cuda_dev, dtype)
            C = torch.empty_like(A)
            for op in ops:
                unary = OPS[op] in (4, 5)
                rc, js = tl.tl_plan_describe(tl.TL_OP_ENTRYWISE, tl.Desc(A, n, pa),
                                             None if unary else tl.Desc(B, n, pb), 0, 0, 0, OPS[op],
                                             tl.Desc(C, n, pc))
                P = json.loads(js)
                assert P["kernel"] == "ew_tile" and P["vec"] == (4 if dtype == "f32" else 2), P
                got, ref = ew_case(tl, cuda_dev, OPS[op], X, Y, pa, pb, pc, dtype)
                np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape,pa,pb,pc", [((7, 3001), (1, 2), (2, 1), (2, 1)),
                                            ((3001, 9), (2, 1), (1, 2), (1, 2)),
                                            ((7, 1001, 5), (2, 3, 1), (3, 2, 1), (1, 2, 3)),
                                            ((33, 31, 6), (1, 2, 3), (2, 1, 3), (1, 2, 3)),
                                            ((13, 4097), (1, 2), (2, 1), (2, 1))])
def test_entrywise_element_tiles_bit_exact(tl, cuda_dev, dtype, shape, pa, pb, pc):
    # odd extents rule out 16-byte vectors: the element tile kernel, whose
    # 1024-element tile takes the shape (16 x 64 .. 128 x 8) that the ragged
    # edges fill best; binary and unary operations, one or both inputs staged
    import json
    X = synth.normal(shape, 3560, dtype=np.float64)
    Y = synth.normal(shape, 3561, dtype=np.float64) + 3.0
    for op in ("add", "div", "copy"):
        A = put(X, pa, cuda_dev, dtype)
        B = put(Y, pb, cuda_dev, dtype)
        C = torch.empty_like(A)
        unary = OPS[op] in (4, 5)
        rc, js = tl.tl_plan_describe(tl.TL_OP_ENTRYWISE, tl.Desc(A, shape, pa),
                                     None if unary else tl.Desc(B, shape, pb), 0, 0, 0, OPS[op],
                                     tl.Desc(C, shape, pc))
        P = json.loads(js)
        if not (unary and pa == pc):
            assert P["kernel"] == "ew_tile" and P["vec"] == 1, P
        got, ref = ew_case(tl, cuda_dev, OPS[op], X, Y, pa, pb, pc, dtype)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_entrywise_shared_fastest_mode_rows_path(tl, cuda_dev, dtype):
    # same fastest mode, the other modes permuted: the per-vector mapper path
    import json
    n = (12, 5, 7, 3)
    X = synth.normal(n, 3500, dtype=np.float64)
    Y = synth.normal(n, 3501, dtype=np.float64)
    for pa, pb, pc in [((1, 3, 2, 4), (1, 2, 3, 4), (1, 4, 3, 2)), ((1, 2, 3, 4), (1, 4, 2, 3), (1, 2, 4, 3))]:
        A = put(X, pa, cuda_dev, dtype)
        B = put(Y, pb, cuda_dev, dtype)
        C = torch.empty_like(A)
        rc, js = tl.tl_plan_describe(tl.TL_OP_ENTRYWISE, tl.Desc(A, n, pa), tl.Desc(B, n, pb),
                                     0, 0, 0, tl.TL_MUL, tl.Desc(C, n, pc))
        assert json.loads(js)["kernel"] == "ew_rows", js
        got, ref = ew_case(tl, cuda_dev, OPS["mul"], X, Y, pa, pb, pc, dtype)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("shape", [(36, 20, 64), (8, 12, 16, 20), (64, 36, 4, 8, 12), (96, 33 * 4, 8),
                                   (4, 4, 4, 4, 4)])
@pytest.mark.parametrize("op", ["add", "div", "copy", "scale"])
def test_entrywise_fp32_mixed_layouts_bit_exact(tl, cuda_dev, shape, op):
    # dense FP32 layout mixes: transposed and direct inputs, ragged tiles, up
    # to 3 batch dims, permuted rows (F, R, F) and (R, F, F): every operand
    # contiguous along mode 1, the rest reversed in B or A
    import json
    p = len(shape)
    g = synth.rng(3600 + p)
    X = synth.normal(shape, 3601, dtype=np.float64)
    Y = synth.normal(shape, 3602, dtype=np.float64) + 3.0
    F, L = synth.first_order(p), synth.last_order(p)
    R = (1,) + tuple(range(p, 1, -1))
    combos = [(F, L, F), (L, F, F), (L, L, F), (F, F, L), (synth.random_layout(p, g), F, F),
              (F, R, F), (R, F, F)]
    for pa, pb, pc in combos:
        A = put(X, pa, cuda_dev, "f32")
        B = put(Y, pb, cuda_dev, "f32")
        C = torch.empty_like(A)
        unary = OPS[op] in (4, 5)
        rc, js = tl.tl_plan_describe(tl.TL_OP_ENTRYWISE, tl.Desc(A, shape, pa),
                                     None if unary else tl.Desc(B, shape, pb), 0, 0, 0, OPS[op],
                                     tl.Desc(C, shape, pc))
        assert rc == 0 and json.loads(js)["kernel"] in ("ew_flat", "ew_tile", "ew_rows",
                                                        "ew_generic"), js
        got, ref = ew_case(tl, cuda_dev, OPS[op], X, Y, pa, pb, pc, "f32")
        np.testing.assert_array_equal(got, ref)


def _padded(X, pi, dev):
    """X in layout pi inside a parent whose fastest mode is padded to a
    multiple of 4 elements: a view with a ragged extent and 16-byte strides."""
    n = X.shape
    pn = list(n)
    pn[pi[0] - 1] = (n[pi[0] - 1] + 3) // 4 * 4
    parent = np.zeros(pn, dtype=np.float32)
    parent[tuple(slice(0, x) for x in n)] = X
    return to_dev(synth.to_memory(parent, pi), dev, "f32"), oracle.strides(tuple(pn), pi)


@pytest.mark.parametrize("shape", [(61, 64, 40), (30, 6, 21, 9), (30, 7, 3, 2, 33), (37, 129)])
@pytest.mark.parametrize("op", ["add", "div", "copy", "scale"])
def test_entrywise_tma_tiles_padded_views_bit_exact(tl, cuda_dev, shape, op):
    # FP32 mixed layouts with a ragged extent whose strides stay multiples of
    # 16 bytes (padded views) take the TMA-staged tile kernel: transposed and
    # direct inputs, ragged tiles, up to 3 batch dims; C's padding keeps its
    # initial value
    import json
    p = len(shape)
    X = synth.normal(shape, 3610, dtype=np.float64).astype(np.float32)
    Y = (synth.normal(shape, 3611, dtype=np.float64) + 3.0).astype(np.float32)
    F, L = synth.first_order(p), synth.last_order(p)
    unary = OPS[op] in (4, 5)
    seen = set()
    for pa, pb, pc in [(F, L, F), (L, F, F), (L, L, F), (F, F, L)]:
        A, wA = _padded(X, pa, cuda_dev)
        B, wB = _padded(Y, pb, cuda_dev)
        C, wC = _padded(np.zeros(shape, dtype=np.float32), pc, cuda_dev)
        C.fill_(-7.0)
        C0 = C.cpu().numpy().astype(np.float64)
        DA, DB, DC = tl.Desc(A, shape, w=wA), tl.Desc(B, shape, w=wB), tl.Desc(C, shape, w=wC)
        rc, js = tl.tl_plan_describe(tl.TL_OP_ENTRYWISE, DA, None if unary else DB, 0, 0, 0,
                                     OPS[op], DC)
        assert rc == 0
        seen.add(json.loads(js)["kernel"])
        tl.check(tl.tl_entrywise(OPS[op], DA, None if unary else DB, -1.5, DC))
        torch.cuda.synchronize()
        ref = oracle.entrywise(OPS[op], shape, A.cpu().numpy(), wA, B.cpu().numpy(), wB, -1.5,
                               C=C0, wC=wC)
        np.testing.assert_array_equal(C.cpu().numpy(), ref.astype(np.float32))
    assert "ew_tma" in seen, seen


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_entrywise_high_order_small_extents_maps_elements(tl, cuda_dev, dtype):
    # order 7, extents 3-13 in unrelated layouts: tiles would be mostly empty,
    # so the planner maps every element; results stay bit-exact
    import json
    n = (13, 3, 7, 5, 4, 6, 3)
    g = synth.rng(3700)
    X = synth.normal(n, 3701, dtype=np.float64)
    Y = synth.normal(n, 3702, dtype=np.float64) + 3.0
    for _ in range(3):
        pa, pb, pc = (synth.random_layout(7, g) for _ in range(3))
        A = put(X, pa, cuda_dev, dtype)
        B = put(Y, pb, cuda_dev, dtype)
        C = torch.empty_like(A)
        rc, js = tl.tl_plan_describe(tl.TL_OP_ENTRYWISE, tl.Desc(A, n, pa), tl.Desc(B, n, pb), 0,
                                     0, 0, tl.TL_ADD, tl.Desc(C, n, pc))
        assert rc == 0 and json.loads(js)["kernel"] in ("ew_generic", "ew_rows", "ew_tma"), js
        for op in ("add", "div"):
            got, ref = ew_case(tl, cuda_dev, OPS[op], X, Y, pa, pb, pc, dtype)
            np.testing.assert_array_equal(got, ref)

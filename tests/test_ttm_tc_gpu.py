"""GPU parity of the tcgen05 tensor-core ttm (Sec. 5.2 Eq. 25) against the FP64
oracle, for TF32, BF16 and split-BF16x3 products with FP32 accumulation.

Bars (relative Frobenius error against the FP64 oracle on the unrounded FP32
inputs): split-BF16x3 <= 1e-5, BF16 <= 1e-2, TF32 <= 1e-2.  Small integers
are exact in BF16 and TF32 and their sums stay below 2^24, so integer-valued
inputs must come out bit-exact in every precision: that pins the kernel's
row / column / k mapping independently of rounding."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import get, put, rel_err, to_dev, ttm_case

pytestmark = pytest.mark.gpu

PREC = {"tf32": 3, "bf16": 4, "bf16x3": 5}
TOL = {"tf32": 1e-2, "bf16": 1e-2, "bf16x3": 1e-5}

# (shape, q, layout): ROW = contraction contiguous, COL = fastest output mode contiguous
SHAPES = [
    ((64, 33, 17), 1, (1, 2, 3)),        # ROW, M = 561 (ragged tile)
    ((96, 40, 8), 1, (1, 2, 3)),         # ROW, nq = 96 (3 stages)
    ((48, 300), 1, (1, 2)),              # ROW, nq = 48 (ragged k stage)
    ((7, 6, 128, 5), 3, (3, 1, 2, 4)),   # ROW via layout: mode 3 fastest
    ((200, 48, 3), 2, (1, 2, 3)),        # COL, inner 200 (ragged), 3 outer
    ((256, 64, 2), 2, (1, 2, 3)),        # COL, exact tiles
    ((128, 100), 2, (1, 2)),             # COL, one outer index, nq = 100
    ((20, 152, 36), 1, (2, 1, 3)),       # COL via layout: mode 2 fastest, q = 1
]
JS = [16, 40, 128, 200, 256, 300, 512]


def plan_kernel(tl, A, n, pi, q, J, C, prec):
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTM, tl.Desc(A, n, pi), None, q, J, prec, 0,
                                 tl.Desc(C, nout, pi))
    assert rc == 0
    return json.loads(js)


@pytest.mark.parametrize("prec", sorted(PREC))
@pytest.mark.parametrize("case", range(len(SHAPES)))
def test_tc_integer_inputs_bit_exact(tl, cuda_dev, prec, case):
    n, q, pi = SHAPES[case]
    g = synth.rng(6000 + case)
    X = synth.integers(n, 6100 + case)
    for J in (JS[case % len(JS)], 48):
        Bm = synth.integers((J, n[q - 1]), 6200 + case + J)
        A = put(X, pi, cuda_dev, "f32")
        C = torch.empty(int(np.prod(n)) // n[q - 1] * J, dtype=torch.float32, device=cuda_dev)
        P = plan_kernel(tl, A, n, pi, q, J, C, PREC[prec])
        assert P["kernel"] == "ttm_tc", P
        got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, "f32", precision=PREC[prec])
        np.testing.assert_array_equal(got, ref)
    assert tl.tl_device_status() == tl.TL_OK


@pytest.mark.parametrize("prec", sorted(PREC))
@pytest.mark.parametrize("J", JS)
def test_tc_random_within_tolerance(tl, cuda_dev, prec, J):
    for case, (n, q, pi) in enumerate(SHAPES):
        X = synth.normal(n, 6300 + case, dtype=np.float64)
        Bm = synth.normal((J, n[q - 1]), 6400 + case, dtype=np.float64)
        got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, "f32", precision=PREC[prec])
        err = rel_err(got, ref)
        assert err <= TOL[prec], (n, q, J, err)
    assert tl.tl_device_status() == tl.TL_OK


@pytest.mark.parametrize("prec", sorted(PREC))
def test_tc_accumulate_and_other_output_layout(tl, cuda_dev, prec):
    n, q, pi = (64, 33, 17), 1, (1, 2, 3)
    X = synth.normal(n, 6500, dtype=np.float64)
    Bm = synth.normal((72, 64), 6501, dtype=np.float64)
    C0 = synth.normal((72, 33, 17), 6502, dtype=np.float64)
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, "f32", precision=PREC[prec],
                        accumulate=True, C0=C0)
    assert rel_err(got, ref) <= TOL[prec]
    # an output layout the tensor-core path does not take falls back to SIMT
    got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, (3, 2, 1), "f32", precision=PREC[prec])
    assert rel_err(got, ref) <= TOL[prec]


def test_tc_bf16x3_beats_bf16_by_orders(tl, cuda_dev):
    n, q, pi = (256, 64, 4), 2, (1, 2, 3)
    X = synth.normal(n, 6600, dtype=np.float64)
    Bm = synth.normal((128, 64), 6601, dtype=np.float64)
    errs = {}
    for prec in PREC:
        got, ref = ttm_case(tl, cuda_dev, X, q, Bm, pi, pi, "f32", precision=PREC[prec])
        errs[prec] = rel_err(got, ref)
    assert errs["bf16x3"] * 100 < errs["bf16"], errs
    assert errs["tf32"] < errs["bf16"], errs


@pytest.fixture(scope="module")
def scale_tensors(cuda_dev):
    case = synth.scale_case()
    n = case.n
    memF = case.mem_first
    X = synth.from_memory(memF, n, synth.first_order(4))
    memL = synth.to_memory(X, synth.last_order(4))
    return case, memF, memL, to_dev(memF, cuda_dev, "f32"), to_dev(memL, cuda_dev, "f32")


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_tc_full_scale_sampled(tl, cuda_dev, scale_tensors, prec):
    case, memF, memL, AF, AL = scale_tensors
    n = case.n
    g = synth.rng(6700)
    C = torch.empty(128 ** 4, dtype=torch.float32, device=cuda_dev)
    for pi, mem, Ad in ((synth.first_order(4), memF, AF), (synth.last_order(4), memL, AL)):
        wA = oracle.strides(n, pi)
        for q in range(1, 5):
            Bm = case.matrices[q - 1]
            Bt = to_dev(Bm.reshape(-1), cuda_dev, "f32")
            P = plan_kernel(tl, Ad, n, pi, q, 128, C, PREC[prec])
            assert P["kernel"] == "ttm_tc", (pi, q, P)
            tl.check(tl.tl_ttm(tl.Desc(Ad, n, pi), Bt, 128, 128, 1, q, tl.Desc(C, n, pi),
                               PREC[prec]))
            torch.cuda.synchronize()
            got = get(C, n, pi)
            idx = np.stack([g.integers(0, x, size=4000) for x in n], axis=1)
            ref = oracle.ttm_at(mem, n, wA, q, Bm.reshape(-1), 128, 1, idx)
            assert rel_err(got[tuple(idx.T)], ref) <= TOL[prec], (pi, q)
    assert tl.tl_device_status() == tl.TL_OK


# The epilogue's store paths: TMA stores of 32 x 32 boxes where C's base and
# strides are 16-byte aligned and nothing accumulates; warp stores otherwise
# (16-byte vectors through a shared-memory transpose, or single elements).
STORE_CASES = [
    # (shape, q, J, C offset in elements, accumulate)
    ((64, 33, 17), 1, 37, 0, False),     # ROW, C rows 37 apart: single elements
    ((200, 48, 3), 2, 37, 0, False),     # COL, TMA boxes clipped at 37 columns
    ((64, 33, 17), 1, 40, 1, False),     # ROW, C base not 16-byte aligned: single elements
    ((200, 48, 3), 2, 40, 1, False),     # COL, C base not 16-byte aligned: single elements
    ((200, 48, 3), 2, 40, 0, True),      # COL, accumulate: vectors along rows
    ((64, 33, 17), 1, 40, 0, True),      # ROW, accumulate: vectors along j
    ((200, 48, 3), 2, 40, 0, False),     # COL, TMA stores (rows past 200 clipped)
    ((64, 33, 17), 1, 40, 0, False),     # ROW, TMA stores (columns past 40 clipped)
]


@pytest.mark.parametrize("prec", sorted(PREC))
@pytest.mark.parametrize("case", range(len(STORE_CASES)))
def test_tc_store_paths_bit_exact(tl, cuda_dev, prec, case):
    n, q, J, off, acc = STORE_CASES[case]
    X = synth.integers(n, 6700 + case)
    Bm = synth.integers((J, n[q - 1]), 6710 + case)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    NC = int(np.prod(nout))
    C0 = synth.integers(nout, 6720 + case) if acc else np.zeros(nout)
    A = put(X, (1, 2, 3), cuda_dev, "f32")
    Bt = to_dev(np.ascontiguousarray(Bm).reshape(-1), cuda_dev, "f32")
    # C at element offset `off` inside a buffer whose other elements hold a sentinel
    buf = torch.full((NC + off + 5,), -7.0, dtype=torch.float32, device=cuda_dev)
    buf[off:off + NC] = torch.from_numpy(synth.to_memory(np.asarray(C0, np.float32),
                                                         (1, 2, 3))).to(cuda_dev)
    Cv = buf[off:off + NC]
    P = plan_kernel(tl, A, n, (1, 2, 3), q, J, Cv, PREC[prec])
    assert P["kernel"] == "ttm_tc", P
    rc = tl.tl_ttm(tl.Desc(A, n), Bt, J, n[q - 1], 1, q, tl.Desc(Cv, nout), PREC[prec], int(acc))
    tl.check(rc, "tl_ttm")
    torch.cuda.synchronize()
    out = buf.cpu().numpy()
    ref = oracle.ttm(synth.to_memory(X, (1, 2, 3)), n, oracle.strides(n), q,
                     np.ascontiguousarray(Bm).reshape(-1), J, n[q - 1], 1,
                     C=synth.to_memory(np.asarray(C0, np.float64), (1, 2, 3)),
                     wC=oracle.strides(nout), accumulate=acc)
    np.testing.assert_array_equal(out[off:off + NC], ref)
    assert np.all(out[:off] == -7.0) and np.all(out[off + NC:] == -7.0)
    assert tl.tl_device_status() == tl.TL_OK


def _round_even(x, drop):
    """FP32 values rounded to nearest, ties to even, keeping 23 - drop
    mantissa bits (drop = 13: TF32, 16: BF16); finite inputs."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> drop) & 1
    b = (b + (1 << (drop - 1)) - 1 + lsb) & ~np.uint64((1 << drop) - 1)
    return b.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("prec,drop", [("tf32", 13), ("bf16", 16)])
def test_tc_conversion_rounds_ties_to_even(tl, cuda_dev, prec, drop):
    # A holds values exactly halfway between two representable TF32 / BF16
    # values (and their neighbours); with B = I each output is one converted
    # element times 1, so C shows the rounding rule: ties go to the even
    # neighbour (1 + 2^-11 -> 1 in TF32, where ties away from zero would give
    # 1 + 2^-10), never away from zero
    n, q, J = (256, 32), 2, 32
    half = np.float32(2.0 ** (-(24 - drop)))          # half an ulp at 1.0
    base = np.array([1.0, 1.0 + 2 * half, -1.0, -(1.0 + 2 * half), 1.5, 3.0], np.float32)
    g = synth.rng(6900)
    vals = np.concatenate([base + half, base - half, base + half / 2, base + 3 * half,
                           base])
    X = g.choice(vals, size=n).astype(np.float32) * np.float32(2.0) ** g.integers(-4, 5, size=n)
    X = X.astype(np.float32)
    A = put(X, (1, 2), cuda_dev, "f32")
    C = torch.empty(n[0] * J, dtype=torch.float32, device=cuda_dev)
    assert plan_kernel(tl, A, n, (1, 2), q, J, C, PREC[prec])["kernel"] == "ttm_tc"
    got, _ = ttm_case(tl, cuda_dev, X, q, np.eye(J), (1, 2), (1, 2), "f32",
                      precision=PREC[prec])
    want = _round_even(X, drop)
    np.testing.assert_array_equal(got, want)
    # the fixture really holds ties: rounding them away from zero differs
    b = np.ascontiguousarray(X).view(np.uint32).astype(np.uint64)
    away = ((b + (1 << (drop - 1))) & ~np.uint64((1 << drop) - 1)).astype(np.uint32)
    assert np.count_nonzero(away.view(np.float32) != want) > 100

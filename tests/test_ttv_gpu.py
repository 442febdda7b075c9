"""GPU parity of tl_ttv (Sec. 5.2 Eq. 24) against the FP64 oracle.

Bars: integer-valued inputs are bit-exact; otherwise the relative Frobenius
error is <= 1e-12 for FP64 and <= 1e-5 for FP32, and every element lies within
the rounding bound of its dot product."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, dot_bound, get, put, rel_err, to_dev, ttv_case

pytestmark = pytest.mark.gpu

EPS = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("seed", range(16))
def test_ttv_random_layouts(tl, cuda_dev, dtype, seed):
    g = synth.rng(1000 + seed)
    p = int(g.integers(2, 7))
    n = tuple(int(x) for x in g.integers(1, 14 if p > 4 else 40, size=p))
    q = int(g.integers(1, p + 1))
    X = synth.uniform(n, 1100 + seed)
    b = synth.uniform((n[q - 1],), 1200 + seed)
    pa, pc = synth.random_layout(p, g), synth.random_layout(p - 1, g)
    acc = bool(g.integers(2))
    C0 = synth.uniform(tuple(x for r, x in enumerate(n) if r != q - 1), 1300 + seed)
    incb = int(g.choice([1, 3]))
    got, ref = ttv_case(tl, cuda_dev, X, q, b, pa, pc, dtype, acc, C0 if acc else None, incb)
    assert got.shape == ref.shape
    assert rel_err(got, ref) <= TOL[dtype]
    Xa = np.abs(X).astype(np.float64)
    bound = dot_bound(Xa, np.abs(b), q, EPS[dtype]) + (np.abs(C0) * EPS[dtype] * 2 if acc else 0)
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ttv_integer_inputs_bit_exact(tl, cuda_dev, dtype):
    g = synth.rng(1400)
    for i in range(8):
        p = int(g.integers(2, 6))
        n = tuple(int(x) for x in g.integers(1, 12, size=p))
        q = int(g.integers(1, p + 1))
        X = synth.integers(n, 1410 + i)
        b = synth.integers((n[q - 1],), 1420 + i)
        got, ref = ttv_case(tl, cuda_dev, X, q, b, synth.random_layout(p, g),
                            synth.random_layout(p - 1, g), dtype)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("shape", [(129, 67, 33), (1000, 257), (5, 3, 7001), (70, 1, 90, 3),
                                   (33, 17, 9, 5, 3), (4097, 3, 2), (128, 1001), (2048, 77),
                                   (256, 3, 700)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ttv_multi_tile_ragged_all_modes(tl, cuda_dev, shape, dtype):
    X = synth.normal(shape, 1500, dtype=np.float64)
    p = len(shape)
    for pi in (synth.first_order(p), synth.last_order(p)):
        for q in range(1, p + 1):
            b = synth.normal((shape[q - 1],), 1501 + q, dtype=np.float64)
            pic = tuple(sorted(r for r in pi if r != q).index(r) + 1 for r in pi if r != q)
            got, ref = ttv_case(tl, cuda_dev, X, q, b, pi, pic, dtype)
            assert rel_err(got, ref) <= TOL[dtype], (pi, q)


@pytest.mark.parametrize("shape,q", [((3, 200000), 2), ((200000, 3), 1), ((2, 2, 50000), 3),
                                     ((6, 40000, 2), 2), ((1, 131072), 2)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ttv_split_k(tl, cuda_dev, shape, q, dtype):
    X = synth.normal(shape, 1600, dtype=np.float64)
    p = len(shape)
    pi = synth.first_order(p)
    nout = tuple(x for r, x in enumerate(shape) if r != q - 1)
    A = put(X, pi, cuda_dev, dtype)
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTV, tl.Desc(A, shape, pi), None, q, 0, 0, 0,
                                 tl.Desc(put(np.zeros(nout), synth.first_order(p - 1), cuda_dev,
                                             dtype), nout))
    assert rc == 0 and json.loads(js)["splits"] > 1, js
    for acc in (False, True):
        b = synth.normal((shape[q - 1],), 1601, dtype=np.float64)
        C0 = synth.normal(nout, 1602, dtype=np.float64) if acc else None
        got, ref = ttv_case(tl, cuda_dev, X, q, b, pi, synth.first_order(p - 1), dtype, acc, C0)
        assert rel_err(got, ref) <= TOL[dtype]


def test_ttv_strided_views(tl, cuda_dev):
    # a view with steps t (Sec. 3.3: n' from Eq. 5, gamma from Eq. 18, w'' = w t)
    for dtype in ("f32", "f64"):
        npar = (9, 8, 11)
        parent = synth.normal(npar, 1700, dtype=np.float64)
        pi = (2, 3, 1)
        w = oracle.strides(npar, pi)
        f, t, l = (1, 0, 2), (2, 3, 2), (8, 7, 10)
        nv, wv, gamma = oracle.view(npar, w, f, t, l)
        mem = synth.to_memory(parent, pi)
        Ad = to_dev(mem, cuda_dev, dtype)
        elem = Ad.element_size()
        for q in (1, 2, 3):
            b = synth.normal((nv[q - 1],), 1701 + q, dtype=np.float64)
            bt = to_dev(b, cuda_dev, dtype)
            nout = tuple(x for r, x in enumerate(nv) if r != q - 1)
            # strided output: every other element of a dense buffer
            Cbig = torch.zeros(2 * int(np.prod(nout)), dtype=Ad.dtype, device=cuda_dev)
            wcv = tuple(2 * x for x in oracle.strides(nout))
            rc = tl.tl_ttv(tl.Desc(Ad.data_ptr() + gamma * elem, nv, w=wv, dtype=Ad.dtype), bt, 1, q,
                           tl.Desc(Cbig, nout, w=wcv), 0)
            tl.check(rc)
            torch.cuda.synchronize()
            ref = oracle.ttv(mem, nv, wv, q, b.astype(np.float32 if dtype == "f32" else np.float64),
                             wC=oracle.strides(nout), offA=gamma)
            got = Cbig.cpu().numpy()[::2]
            assert rel_err(got, ref) <= TOL[dtype]
            assert np.all(Cbig.cpu().numpy()[1::2] == 0)


def test_ttv_small_case_fp64(tl, cuda_dev):
    case = synth.small_case()
    got, ref = ttv_case(tl, cuda_dev, case.X, case.q_ttv, case.b, (1, 2, 3), (1, 2), "f64")
    assert rel_err(got, ref) <= 1e-12


def test_ttv_extent_one_and_unit_contraction(tl, cuda_dev):
    for n, q in [((1, 1, 5), 3), ((7, 1), 2), ((1, 9), 1), ((3, 4, 1), 3), ((1, 1), 1)]:
        X = synth.normal(n, 1800, dtype=np.float64)
        b = synth.normal((n[q - 1],), 1801, dtype=np.float64)
        p = len(n)
        got, ref = ttv_case(tl, cuda_dev, X, q, b, synth.last_order(p), synth.first_order(p - 1),
                            "f64")
        assert rel_err(got, ref) <= 1e-12


def test_ttv_rejects_bad_calls_without_launching(tl, cuda_dev):
    A = torch.zeros(24, device=cuda_dev)
    C = torch.zeros(8, device=cuda_dev)
    b = torch.zeros(3, device=cuda_dev)
    assert tl.tl_ttv(tl.Desc(A, (2, 3, 4)), b, 1, 4, tl.Desc(C, (2, 4))) == tl.TL_EINVAL
    assert tl.tl_ttv(tl.Desc(A, (2, 3, 4)), b, 1, 2, tl.Desc(A, (2, 4))) == tl.TL_EINVAL
    assert tl.tl_ttv(tl.Desc(A, (2, 3, 4)), 0, 1, 2, tl.Desc(C, (2, 4))) == tl.TL_EINVAL


@pytest.fixture(scope="module")
def scale_tensors(cuda_dev):
    """The 128^4 FP32 workload in first-order and last-order layouts."""
    case = synth.scale_case()
    n = case.n
    memF = case.mem_first
    X = synth.from_memory(memF, n, synth.first_order(4))
    memL = synth.to_memory(X, synth.last_order(4))
    return case, memF, memL, to_dev(memF, cuda_dev, "f32"), to_dev(memL, cuda_dev, "f32")


def test_ttv_full_scale_sampled(tl, cuda_dev, scale_tensors):
    case, memF, memL, AF, AL = scale_tensors
    n = case.n
    g = synth.rng(1900)
    for pi, mem, Ad in ((synth.first_order(4), memF, AF), (synth.last_order(4), memL, AL)):
        wA = oracle.strides(n, pi)
        for q in range(1, 5):
            nout = tuple(x for r, x in enumerate(n) if r != q - 1)
            pic = tuple(sorted(r for r in pi if r != q).index(r) + 1 for r in pi if r != q)
            C = torch.empty(int(np.prod(nout)), dtype=torch.float32, device=cuda_dev)
            bt = to_dev(case.vectors[q - 1], cuda_dev, "f32")
            tl.check(tl.tl_ttv(tl.Desc(Ad, n, pi), bt, 1, q, tl.Desc(C, nout, pic)))
            torch.cuda.synchronize()
            got = get(C, nout, pic)
            idx = np.stack([g.integers(0, x, size=3000) for x in nout], axis=1)
            ref = oracle.ttv_at(mem, n, wA, q, case.vectors[q - 1], idx)
            sample = got[tuple(idx.T)]
            assert rel_err(sample, ref) <= 1e-5, (pi, q)


def test_ttv_staged_row_kernel_selected_and_exact_on_integers(tl, cuda_dev):
    # dense rows (q fastest), n_q a multiple of 128: the bulk-copy staged path
    for dtype, n in (("f32", (128, 3001)), ("f64", (256, 999)), ("f32", (2048, 50))):
        X = synth.integers(n, 1950)
        b = synth.integers((n[0],), 1951)
        got, ref = ttv_case(tl, cuda_dev, X, 1, b, (1, 2), (1,), dtype)
        np.testing.assert_array_equal(got, ref)
    assert tl.tl_device_status() == tl.TL_OK


def test_nvtx_ranges_do_not_change_results(tl, cuda_dev):
    # TL_NVTX=1 wraps every entry point in an NVTX range (read once per
    # process), so the check runs in a child process
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    code = (
        "import sys; sys.path[:0] = [%r, %r]\n"
        "import numpy as np, torch, oracle, synth\n"
        "import paper_1711_10912_gb300 as tl\n"
        "tl.load_library()\n"
        "from gpu_util import ttv_case, ttm_case, rel_err\n"
        "dev = torch.device('cuda', 0)\n"
        "X = synth.uniform((33, 17, 9), 4600)\n"
        "got, ref = ttv_case(tl, dev, X, 2, synth.uniform((17,), 4601), (1, 2, 3), (2, 1), 'f64')\n"
        "assert rel_err(got, ref) <= 1e-12\n"
        "got, ref = ttm_case(tl, dev, X, 3, synth.uniform((5, 9), 4602), (3, 1, 2), (1, 2, 3), 'f64')\n"
        "assert rel_err(got, ref) <= 1e-12\n"
        "print('ok')\n" % (here, os.path.dirname(here)))
    res = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, TL_NVTX="1"),
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and res.stdout.strip().endswith("ok"), res.stderr[-2000:]

"""tl_ttv_noalloc: the ttv entry point for callers that cannot let a library
allocate device memory (runtimes that own all device memory under their own
budget, and latency-critical loops where cudaMalloc / cudaFree would
synchronise the device).  It keeps split-K partial sums in a static device
array instead of a workspace.

Checked here through the C ABI on two calls in a row, with shapes whose plan
splits the contraction and therefore uses the scratch: the output must be
bit-identical to tl_ttv's (the workspace-based entry point runs the same plan
and kernels, and the split sums are added in a fixed order) and within the
stated tolerance of the FP64 oracle; a call must leave the device's free
memory unchanged where tl_ttv's first call on a new stream allocates; and a
call whose partial sums would not fit is rejected.  This file is collected
last on purpose."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, put, rel_err

pytestmark = pytest.mark.gpu

CASES = [((3, 200000), 2, "f32"), ((100000, 64), 2, "f32"), ((50000, 64), 2, "f64"),
         ((2, 2, 50000), 3, "f64")]


def _plan(tl, A, n, q, C, nout):
    rc, js = tl.tl_plan_describe(tl.TL_OP_TTV, tl.Desc(A, n), None, q, 0, 0, 0, tl.Desc(C, nout))
    assert rc == 0
    return json.loads(js)


@pytest.mark.parametrize("n,q,dtype", CASES)
def test_noalloc_matches_tl_ttv_on_two_calls(tl, cuda_dev, n, q, dtype):
    p = len(n)
    nout = tuple(x for r, x in enumerate(n) if r != q - 1)
    X = synth.normal(n, 5000, dtype=np.float64)
    A = put(X, synth.first_order(p), cuda_dev, dtype)
    b = put(synth.normal((n[q - 1],), 5001, dtype=np.float64), (1,), cuda_dev, dtype)
    C_ref = torch.empty(int(np.prod(nout)), dtype=A.dtype, device=cuda_dev)
    C_na = torch.full_like(C_ref, float("nan"))
    P = _plan(tl, A, n, q, C_ref, nout)
    scratch = P["splits"] * P["nout"] * A.element_size()
    assert P["splits"] > 1 and scratch <= tl.TL_TTV_NOALLOC_SCRATCH_BYTES, P
    tl.check(tl.tl_ttv(tl.Desc(A, n), b, 1, q, tl.Desc(C_ref, nout)), "tl_ttv")
    mem = synth.to_memory(np.asarray(X, dtype=np.float32 if dtype == "f32" else np.float64),
                          synth.first_order(p))
    ref_oracle = oracle.ttv(mem, n, oracle.strides(n), q, b.cpu().numpy())
    for call in range(2):
        C_na.fill_(float("nan"))
        tl.check(tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, q, tl.Desc(C_na, nout)), "tl_ttv_noalloc")
        torch.cuda.synchronize()
        got, ref = C_na.cpu().numpy(), C_ref.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}: output not fully written"
        np.testing.assert_array_equal(got, ref, err_msg=f"call {call}")
        assert rel_err(got, ref_oracle) <= TOL[dtype], f"call {call}"


def test_noalloc_accumulate_matches(tl, cuda_dev):
    n, q = (100000, 64), 2
    X = synth.normal(n, 5100, dtype=np.float64)
    A = put(X, (1, 2), cuda_dev, "f32")
    b = put(synth.normal((64,), 5101, dtype=np.float64), (1,), cuda_dev, "f32")
    C0 = put(synth.normal((n[0],), 5102, dtype=np.float64), (1,), cuda_dev, "f32")
    C_ref, C_na = C0.clone(), C0.clone()
    tl.check(tl.tl_ttv(tl.Desc(A, n), b, 1, q, tl.Desc(C_ref, (n[0],)), 1))
    tl.check(tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, q, tl.Desc(C_na, (n[0],)), 1))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C_na.cpu().numpy(), C_ref.cpu().numpy())
    mem = synth.to_memory(X.astype(np.float32), (1, 2))
    ref = oracle.ttv(mem, n, oracle.strides(n), q, b.cpu().numpy(), C=C0.cpu().numpy(),
                     wC=(1,), accumulate=True)
    assert rel_err(C_na.cpu().numpy(), ref) <= TOL["f32"]


def test_noalloc_leaves_device_memory_unchanged(tl, cuda_dev):
    # about 3 MiB of FP32 partial sums (under the 4 MiB scratch); each call
    # runs on a stream of its own, which tl_ttv has never used, so tl_ttv has
    # to allocate a workspace there while tl_ttv_noalloc must not allocate
    n, q = (200000, 64), 2
    A = torch.randn(n[0] * n[1], dtype=torch.float32, device=cuda_dev)
    b = torch.randn(n[1], dtype=torch.float32, device=cuda_dev)
    C1 = torch.empty(n[0], dtype=torch.float32, device=cuda_dev)
    C2 = torch.empty_like(C1)
    P = _plan(tl, A, n, q, C1, (n[0],))
    need = P["splits"] * P["nout"] * 4
    assert 3 << 20 <= need <= tl.TL_TTV_NOALLOC_SCRATCH_BYTES, P
    s_na, s_ws = torch.cuda.Stream(), torch.cuda.Stream()
    # one call first, so the library's kernels and the scratch array are loaded
    tl.check(tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, q, tl.Desc(C1, (n[0],))))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    tl.check(tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, q, tl.Desc(C1, (n[0],)), 0,
                               s_na.cuda_stream))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    tl.check(tl.tl_ttv(tl.Desc(A, n), b, 1, q, tl.Desc(C2, (n[0],)), 0, s_ws.cuda_stream))
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert free2 <= free1 - need, (free1, free2)     # the check can see an allocation
    np.testing.assert_array_equal(C1.cpu().numpy(), C2.cpu().numpy())


def test_noalloc_rejects_calls_beyond_the_static_scratch(tl, cuda_dev):
    # 400000 outputs split 4 ways need 6.4 MB of FP32 partials > 4 MiB
    n, q = (400000, 64), 2
    A = torch.zeros(n[0] * n[1], dtype=torch.float32, device=cuda_dev)
    b = torch.ones(64, dtype=torch.float32, device=cuda_dev)
    C = torch.full((n[0],), 7.0, dtype=torch.float32, device=cuda_dev)
    P = _plan(tl, A, n, q, C, (n[0],))
    assert P["splits"] * P["nout"] * 4 > tl.TL_TTV_NOALLOC_SCRATCH_BYTES, P
    assert tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, q, tl.Desc(C, (n[0],))) == tl.TL_ENOMEM
    torch.cuda.synchronize()
    assert torch.all(C == 7.0)          # nothing was enqueued
    tl.check(tl.tl_ttv(tl.Desc(A, n), b, 1, q, tl.Desc(C, (n[0],))))
    torch.cuda.synchronize()
    assert torch.all(C == 0.0)


def test_noalloc_without_split_needs_no_scratch(tl, cuda_dev):
    # a contraction of 16 is too short to split, so no scratch is used
    n, q = (64, 16, 64), 2
    X = synth.normal(n, 5200, dtype=np.float64)
    A = put(X, (1, 2, 3), cuda_dev, "f64")
    b = put(synth.normal((16,), 5201, dtype=np.float64), (1,), cuda_dev, "f64")
    C_ref = torch.empty(64 * 64, dtype=torch.float64, device=cuda_dev)
    C_na = torch.empty_like(C_ref)
    assert _plan(tl, A, n, q, C_ref, (64, 64))["splits"] == 1
    tl.check(tl.tl_ttv(tl.Desc(A, n), b, 1, q, tl.Desc(C_ref, (64, 64))))
    tl.check(tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, q, tl.Desc(C_na, (64, 64))))
    torch.cuda.synchronize()
    assert rel_err(C_na.cpu().numpy(), C_ref.cpu().numpy()) <= TOL["f64"]

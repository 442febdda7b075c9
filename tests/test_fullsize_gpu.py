"""Full-size parity in the launch configurations the benchmark times.

- The 512^3 precision workload (mode-3 slices scaled by 10^U(-3,3)): ttm by a
  512x512 and a truncated 64x512 matrix along every mode in FP32 (SIMT),
  BF16, TF32 and split-BF16x3, and the all-modes Tucker projection to 64^3, checked on
  sampled outputs against the FP64 oracle.
- The 4096-operation batch (orders 3-6, extents log-uniform in [4, 64],
  random layouts and modes): one persistent, graph-captured, autotuned launch
  against the per-call path, plus whole-output oracle checks of a sample of
  the operations."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

TOL = {3: 1e-2, 4: 1e-2, 5: 1e-5, 2: 1e-5}


@pytest.fixture(scope="module")
def precision_case(cuda_dev):
    n, mem, B, Bt, U = synth.precision_case()
    return n, mem, B, Bt, U, torch.from_numpy(mem).to(cuda_dev)


@pytest.mark.parametrize("which", ["x512", "x64"])
def test_precision_study_all_modes(tl, cuda_dev, precision_case, which):
    n, mem, B, Bt, U, A = precision_case
    Bm = B if which == "x512" else Bt
    J = Bm.shape[0]
    Bd = torch.from_numpy(np.ascontiguousarray(Bm).reshape(-1)).to(cuda_dev)
    w = oracle.strides(n)
    g = synth.rng(9000 + J)
    for q in (1, 2, 3):
        nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
        C = torch.empty(int(np.prod(nout)), dtype=torch.float32, device=cuda_dev)
        idx = np.stack([g.integers(0, x, size=2000) for x in nout], axis=1)
        ref = oracle.ttm_at(mem, n, w, q, Bm.reshape(-1), 512, 1, idx)
        for prec in (2, 3, 4, 5):
            tl.check(tl.tl_ttm(tl.Desc(A, n), Bd, J, 512, 1, q, tl.Desc(C, nout), prec))
            torch.cuda.synchronize()
            got = synth.from_memory(C.cpu().numpy(), nout, (1, 2, 3))[tuple(idx.T)]
            assert rel_err(got, ref) <= TOL[prec], (which, q, prec)
    assert tl.tl_device_status() == tl.TL_OK


def test_tucker_projection_steps(tl, cuda_dev, precision_case):
    n, mem, B, Bt, U, A = precision_case
    cur, cur_n, cur_mem = A, n, mem
    g = synth.rng(9100)
    for q in (1, 2, 3):
        Ud = torch.from_numpy(np.ascontiguousarray(U[q - 1]).reshape(-1)).to(cuda_dev)
        nout = tuple(64 if r == q - 1 else x for r, x in enumerate(cur_n))
        C = torch.empty(int(np.prod(nout)), dtype=torch.float32, device=cuda_dev)
        tl.check(tl.tl_ttm(tl.Desc(cur, cur_n), Ud, 64, 512, 1, q, tl.Desc(C, nout), 5))
        torch.cuda.synchronize()
        idx = np.stack([g.integers(0, x, size=2000) for x in nout], axis=1)
        ref = oracle.ttm_at(cur_mem, cur_n, oracle.strides(cur_n), q, U[q - 1].reshape(-1), 512,
                            1, idx)
        out_mem = C.cpu().numpy()
        got = synth.from_memory(out_mem, nout, (1, 2, 3))[tuple(idx.T)]
        assert rel_err(got, ref) <= 1e-5, q
        cur, cur_n, cur_mem = C, nout, out_mem
    assert cur_n == (64, 64, 64)


def test_batch_4096_persistent_matches_per_call_and_oracle(tl, cuda_dev):
    units = synth.batch_units(4096)
    keep, ops, calls, outs, hostcheck = [], [], [], [], []
    g = synth.rng(9200)
    sample = set(int(x) for x in g.choice(4096, size=24, replace=False))
    for i, u in enumerate(units):
        n, pi, q = u.n, u.pi, u.q
        N = int(np.prod(n))
        A = synth.device_normal(torch, N, 50_000 + 7 * i, torch.float32, cuda_dev)
        DA = tl.Desc(A, n, pi)
        if u.op == "ttv":
            nout = tuple(x for r, x in enumerate(n) if r != q - 1)
            pic = tuple(sorted(r for r in pi if r != q).index(r) + 1 for r in pi if r != q)
            b = synth.device_normal(torch, n[q - 1], 50_001 + 7 * i, torch.float32, cuda_dev)
            C = torch.empty(N // n[q - 1], dtype=torch.float32, device=cuda_dev)
            DC = tl.Desc(C, nout, pic)
            ops.append(tl.make_op(tl.TL_OP_TTV, DA, DC, q=q, vec=b))
            calls.append((tl.tl_ttv, (DA, b, 1, q, DC, 0)))
            keep += [A, b, C, DA, DC]
            if i in sample:
                hostcheck.append((C, lambda A=A, b=b, n=n, pi=pi, q=q, nout=nout, pic=pic:
                                  oracle.ttv(A.cpu().numpy(), n, oracle.strides(n, pi), q,
                                             b.cpu().numpy(), wC=oracle.strides(nout, pic))))
        else:
            J = u.J
            nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
            B = synth.device_normal(torch, J * n[q - 1], 50_002 + 7 * i, torch.float32, cuda_dev)
            C = torch.empty(N // n[q - 1] * J, dtype=torch.float32, device=cuda_dev)
            DC = tl.Desc(C, nout, pi)
            ops.append(tl.make_op(tl.TL_OP_TTM, DA, DC, q=q, vec=B, J=J, ldb_row=n[q - 1],
                                  ldb_col=1))
            calls.append((tl.tl_ttm, (DA, B, J, n[q - 1], 1, q, DC, 0, 0)))
            keep += [A, B, C, DA, DC]
            if i in sample:
                hostcheck.append((C, lambda A=A, B=B, n=n, pi=pi, q=q, J=J, nout=nout:
                                  oracle.ttm(A.cpu().numpy(), n, oracle.strides(n, pi), q,
                                             B.cpu().numpy(), J, n[q - 1], 1,
                                             wC=oracle.strides(nout, pi))))
        outs.append(C)
    rc, batch = tl.tl_batch_create(ops, tl.TL_BATCH_TUNE | tl.TL_BATCH_GRAPH)
    tl.check(rc)
    try:
        tl.check(tl.tl_batch_run(batch))
        torch.cuda.synchronize()
        persistent = [c.clone() for c in outs]
        for C, ref_fn in hostcheck:
            assert rel_err(C.cpu().numpy(), ref_fn()) <= 1e-5
        for fn, args in calls:
            tl.check(fn(*args))
        torch.cuda.synchronize()
        for a, b in zip(persistent, outs):
            d = float(torch.linalg.vector_norm((a - b).double()))
            assert d <= 1e-5 * float(torch.linalg.vector_norm(b.double())) + 1e-30
    finally:
        tl.tl_batch_destroy(batch)

"""Kernels whose shared memory exceeds the default 48 KB limit need a
per-function attribute, and CUDA keeps that attribute per device.  With two or
more GPUs visible, the staged-row ttv, the TMA entrywise add, the tensor-core
ttm, the FP32 SIMT ttm and tl_ttv_noalloc run on device 0 and then on device 1
in the same process and must match the FP64 oracle on both (skipped with one
GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def test_each_device_gets_its_own_shared_memory_opt_in(tl, cuda_dev):
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    n = (512, 2000)
    X = synth.normal(n, 7700, dtype=np.float64).astype(np.float32)
    Y = synth.normal(n, 7701, dtype=np.float64).astype(np.float32)
    bv = synth.normal((512,), 7702, dtype=np.float64).astype(np.float32)
    Bm = synth.normal((64, 512), 7703, dtype=np.float64).astype(np.float32)
    memF = synth.to_memory(X, (1, 2))
    memYL = synth.to_memory(Y, (2, 1))
    ref_ttv = oracle.ttv(memF, n, oracle.strides(n), 1, bv)
    ref_add = oracle.entrywise(oracle.OP_ADD, n, memF, oracle.strides(n), memYL,
                               oracle.strides(n, (2, 1)))
    ref_ttm = oracle.ttm(memF, n, oracle.strides(n), 1, Bm.reshape(-1), 64, 512, 1)
    for d in (0, 1):
        dev = torch.device("cuda", d)
        with torch.cuda.device(dev):
            A = torch.from_numpy(memF).to(dev)
            AL = torch.from_numpy(memYL).to(dev)
            b = torch.from_numpy(bv).to(dev)
            B = torch.from_numpy(Bm.reshape(-1).copy()).to(dev)
            C = torch.empty(n[1], dtype=torch.float32, device=dev)
            tl.check(tl.tl_ttv(tl.Desc(A, n), b, 1, 1, tl.Desc(C, (n[1],))))
            Cn = torch.empty_like(C)
            tl.check(tl.tl_ttv_noalloc(tl.Desc(A, n), b, 1, 1, tl.Desc(Cn, (n[1],))))
            S = torch.empty_like(A)
            tl.check(tl.tl_entrywise(tl.TL_ADD, tl.Desc(A, n), tl.Desc(AL, n, (2, 1)), 0.0,
                                     tl.Desc(S, n)))
            outs = {}
            for prec in (tl.TL_P_BF16X3, tl.TL_P_F32):
                T = torch.empty(64 * n[1], dtype=torch.float32, device=dev)
                tl.check(tl.tl_ttm(tl.Desc(A, n), B, 64, 512, 1, 1, tl.Desc(T, (64, n[1])), prec,
                                   0))
                outs[prec] = T
            torch.cuda.synchronize(dev)
            assert rel_err(C.cpu().numpy(), ref_ttv) <= 1e-5, d
            np.testing.assert_array_equal(Cn.cpu().numpy(), C.cpu().numpy())
            np.testing.assert_array_equal(S.cpu().numpy(), ref_add.astype(np.float32))
            for prec, T in outs.items():
                assert rel_err(T.cpu().numpy(), ref_ttm) <= 1e-5, (d, prec)
            assert tl.tl_device_status() == tl.TL_OK

"""Tensors of more than 2^31 elements: order 3, FP32, 2048 x 1024 x 1025 =
2,149,580,800 elements (8.6 GB each).  Element offsets no longer fit 32 bits
(output indices of ttv / ttm still do), so every kernel that decodes indices
in 32-bit arithmetic when they fit must still form 64-bit offsets, and the
flat and TMA entrywise paths must walk 64-bit element counts.

Checked on sampled outputs against the FP64 oracle (Sec. 5.2 Eqs. 24-25,
Sec. 5.1 Eq. 23).  The oracle's inputs are the sampled fibers and elements
gathered by torch indexing from the seeded device tensors, not by this
library; it evaluates them as a small (n_q x samples) tensor."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

N_EXT = (2048, 1024, 1025)
N = int(np.prod(N_EXT))
S = 512                       # sampled outputs per check


@pytest.fixture(scope="module")
def big(cuda_dev):
    free, _ = torch.cuda.mem_get_info(cuda_dev)
    if free < 5 * N * 4 + (2 << 30):
        pytest.skip("needs about 45 GB of free device memory")
    assert N > 2 ** 31
    A = synth.device_normal(torch, N, 3100, torch.float32, cuda_dev)
    yield A
    del A
    torch.cuda.empty_cache()


def _gather(X, offs):
    """FP64 host copy of X's elements at the given (int64) element offsets."""
    t = torch.from_numpy(np.ascontiguousarray(offs, dtype=np.int64).reshape(-1)).to(X.device)
    return X[t].double().cpu().numpy()


def _fibers(A, n, w, q, idx_rest):
    """Mode-q fibers of A through the sampled index tuples of the other modes
    (samples x n_q, FP64)."""
    rest = [r for r in range(len(n)) if r != q - 1]
    base = np.zeros(idx_rest.shape[0], dtype=np.int64)
    for j, r in enumerate(rest):
        base += idx_rest[:, j].astype(np.int64) * w[r]
    nq = n[q - 1]
    offs = base[:, None] + np.arange(nq, dtype=np.int64)[None, :] * w[q - 1]
    return _gather(A, offs).reshape(idx_rest.shape[0], nq)


def test_ttv_beyond_2_31_elements(tl, cuda_dev, big):
    A, n = big, N_EXT
    w = oracle.strides(n)
    g = synth.rng(3110)
    for q in (1, 2, 3):
        nq = n[q - 1]
        b = np.asarray(synth.uniform((nq,), 3120 + q), np.float32)
        bd = torch.from_numpy(b).to(cuda_dev)
        nout = tuple(x for r, x in enumerate(n) if r != q - 1)
        C = torch.empty(N // nq, dtype=torch.float32, device=cuda_dev)
        tl.check(tl.tl_ttv(tl.Desc(A, n), bd, 1, q, tl.Desc(C, nout), 0))
        torch.cuda.synchronize()
        idx = np.stack([g.integers(0, x, size=S) for x in nout], axis=1)
        fib = _fibers(A, n, w, q, idx)
        # the fibers as an (n_q, S) first-order tensor, contracted along mode 1
        ref = oracle.ttv(fib.reshape(-1), (nq, S), (1, nq), 1, b.astype(np.float64))
        wc = oracle.strides(nout)
        got = _gather(C, idx[:, 0] * wc[0] + idx[:, 1] * wc[1])
        assert rel_err(got, ref) <= 1e-5, q
        del C
    assert tl.tl_device_status() == tl.TL_OK


@pytest.mark.parametrize("q,prec", [(1, 5), (2, 5), (3, 5), (2, 2)])
def test_ttm_beyond_2_31_elements(tl, cuda_dev, big, q, prec):
    A, n = big, N_EXT
    w = oracle.strides(n)
    g = synth.rng(3130 + 10 * q + prec)
    J, nq = 64, n[q - 1]
    Bm = np.asarray(synth.uniform((J, nq), 3140 + q), np.float32)
    Bd = torch.from_numpy(np.ascontiguousarray(Bm).reshape(-1)).to(cuda_dev)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    C = torch.empty(N // nq * J, dtype=torch.float32, device=cuda_dev)
    tl.check(tl.tl_ttm(tl.Desc(A, n), Bd, J, nq, 1, q, tl.Desc(C, nout), prec, 0))
    torch.cuda.synchronize()
    idx = np.stack([g.integers(0, x, size=S) for x in nout], axis=1)
    rest = [r for r in range(3) if r != q - 1]
    fib = _fibers(A, n, w, q, idx[:, rest])
    # every row of B against every sampled fiber: a (J, S) first-order output
    allj = oracle.ttm(fib.reshape(-1), (nq, S), (1, nq), 1, Bm.reshape(-1).astype(np.float64),
                      J, nq, 1)
    ref = allj[idx[:, q - 1] + J * np.arange(S)]
    wc = oracle.strides(nout)
    got = _gather(C, sum(idx[:, r].astype(np.int64) * wc[r] for r in range(3)))
    assert rel_err(got, ref) <= 1e-5, (q, prec)
    del C
    assert tl.tl_device_status() == tl.TL_OK


def test_entrywise_beyond_2_31_elements(tl, cuda_dev, big):
    A, n = big, N_EXT
    F, L = (1, 2, 3), (3, 2, 1)
    wF, wL = oracle.strides(n, F), oracle.strides(n, L)
    g = synth.rng(3150)
    idx = np.stack([g.integers(0, x, size=4 * S) for x in n], axis=1)
    offF = sum(idx[:, r].astype(np.int64) * wF[r] for r in range(3))
    offL = sum(idx[:, r].astype(np.int64) * wL[r] for r in range(3))
    Bf = synth.device_normal(torch, N, 3160, torch.float32, cuda_dev)
    C = torch.empty(N, dtype=torch.float32, device=cuda_dev)
    a = _gather(A, offF)
    b = _gather(Bf, offF)
    ones = (1,)
    expect = oracle.entrywise(oracle.OP_ADD, (4 * S,), a, ones, b, ones).astype(np.float32)
    # same layout: the flat kernel over 2^31+ elements
    tl.check(tl.tl_entrywise(tl.TL_ADD, tl.Desc(A, n, F), tl.Desc(Bf, n, F), 1.0,
                             tl.Desc(C, n, F)))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_gather(C, offF).astype(np.float32), expect)
    # B in last-order layout (a torch relayout of the same values): the
    # mixed-layout kernel
    Bl = Bf.view(n[2], n[1], n[0]).permute(2, 1, 0).contiguous().view(-1)
    del Bf
    np.testing.assert_array_equal(_gather(Bl, offL), b)
    C.fill_(float("nan"))
    tl.check(tl.tl_entrywise(tl.TL_ADD, tl.Desc(A, n, F), tl.Desc(Bl, n, L), 1.0,
                             tl.Desc(C, n, F)))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_gather(C, offF).astype(np.float32), expect)
    # no element of C left unwritten
    assert not bool(torch.isnan(C).any())
    del Bl, C
    torch.cuda.empty_cache()
    assert tl.tl_device_status() == tl.TL_OK

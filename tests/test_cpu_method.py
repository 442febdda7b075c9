"""The plain CPU method (the paper's recursive ttv, ttm and transform,
restated in cpu_method/recursive.cpp) is a timed baseline; these host tests
check it against the FP64 oracle on small tensors in random layouts, for
every mode, and its bounded-sample mode (only the first indices of the
outermost recursion level are computed)."""
import numpy as np
import pytest

import cpu_method
import oracle
import synth
from gpu_util import rel_err


@pytest.mark.parametrize("seed", range(6))
def test_recursive_ttv_ttm_transform_match_the_oracle(seed):
    g = synth.rng(8800 + seed)
    p = int(g.integers(2, 6))
    n = tuple(int(x) for x in g.integers(1, 9, size=p))
    X = synth.normal(n, 8810 + seed, dtype=np.float64).astype(np.float32)
    pi = synth.random_layout(p, g)
    mem = synth.to_memory(X, pi)
    w = oracle.strides(n, pi)
    for q in range(1, p + 1):
        nout = tuple(x for r, x in enumerate(n) if r != q - 1)
        pic = synth.random_layout(p - 1, g)
        wC = oracle.strides(nout, pic)
        wC_by_A = [0] * p
        for r, c in zip([r for r in range(p) if r != q - 1], range(p - 1)):
            wC_by_A[r] = wC[c]
        b = synth.normal((n[q - 1],), 8820 + q, dtype=np.float64).astype(np.float32)
        C = np.zeros(int(np.prod(nout)), np.float32)
        cpu_method.ttv(mem, n, w, q, b, C, wC_by_A, nthreads=2)
        ref = oracle.ttv(mem, n, w, q, b, wC=wC)
        assert rel_err(C, ref) <= 1e-5, (n, pi, q)
        J = int(g.integers(1, 6))
        Bm = synth.normal((J, n[q - 1]), 8830 + q, dtype=np.float64).astype(np.float32)
        ncm = tuple(J if r == q - 1 else x for r, x in enumerate(n))
        wCm = oracle.strides(ncm, pi)
        Cm = np.zeros(int(np.prod(ncm)), np.float32)
        cpu_method.ttm(mem, n, w, q, Bm.reshape(-1), J, n[q - 1], 1, Cm, wCm, nthreads=2)
        refm = oracle.ttm(mem, n, w, q, Bm.reshape(-1), J, n[q - 1], 1, wC=wCm)
        assert rel_err(Cm, refm) <= 1e-5, (n, pi, q, J)
    Y = synth.normal(n, 8840 + seed, dtype=np.float64).astype(np.float32)
    piB, piC = synth.random_layout(p, g), synth.random_layout(p, g)
    memB = synth.to_memory(Y, piB)
    wB, wCe = oracle.strides(n, piB), oracle.strides(n, piC)
    Ce = np.zeros(int(np.prod(n)), np.float32)
    cpu_method.transform(0, mem, w, memB, wB, Ce, wCe, n, nthreads=2)
    refe = oracle.entrywise(oracle.OP_ADD, n, mem, w, memB, wB, wC=wCe)
    np.testing.assert_array_equal(Ce, refe.astype(np.float32))


def test_sample_computes_only_the_first_slices():
    n = (6, 5, 4)
    X = synth.normal(n, 8900, dtype=np.float64).astype(np.float32)
    mem = synth.to_memory(X, (1, 2, 3))
    w = oracle.strides(n)
    Bm = synth.normal((3, 5), 8901, dtype=np.float64).astype(np.float32)
    nout = (6, 3, 4)
    C = np.full(int(np.prod(nout)), np.nan, np.float32)
    cpu_method.ttm(mem, n, w, 2, Bm.reshape(-1), 3, 5, 1, C, oracle.strides(nout), count=2)
    Cl = synth.from_memory(C, nout, (1, 2, 3))
    ref = synth.from_memory(oracle.ttm(mem, n, w, 2, Bm.reshape(-1), 3, 5, 1), nout, (1, 2, 3))
    assert rel_err(Cl[:, :, :2], ref[:, :, :2]) <= 1e-6
    assert np.all(np.isnan(Cl[:, :, 2:]))
    assert cpu_method.threads() >= 1

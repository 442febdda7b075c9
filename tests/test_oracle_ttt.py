"""Pins for the oracle's transposition (Table 3, transpose) and (q, phi, psi)-mode
tensor-tensor multiplication (Sec. 5.2): numpy transpose / einsum on random
tensors in random layouts, brute force on tiny inputs, the special cases the
paper names (ttv, ttm, inner and outer product) and the worked example's
shapes."""
import itertools

import numpy as np
import pytest

import oracle
import synth

LETTERS = "abcdefghijklmnop"


def _mem(X, pi):
    return synth.to_memory(X, pi), oracle.strides(X.shape, pi)


def _logical(buf, n, w):
    """Logical array of a strided FP64 buffer (via numpy strides)."""
    if not n:
        return np.asarray(buf[0])
    return np.lib.stride_tricks.as_strided(np.asarray(buf, dtype=np.float64), shape=n,
                                           strides=[8 * x for x in w]).copy()


# ------------------------------------------------------------- transpose ---

def test_transpose_matches_numpy_every_tau(seed=0):
    g = synth.rng(30 + seed)
    n = (3, 5, 2, 4)
    X = synth.uniform(n, 31 + seed)
    for tau in itertools.permutations((1, 2, 3, 4)):
        pa, pc = synth.random_layout(4, g), synth.random_layout(4, g)
        mem, w = _mem(X, pa)
        nc = tuple(n[t - 1] for t in tau)
        wc = oracle.strides(nc, pc)
        buf, got_n = oracle.transpose(mem, n, w, tau, wC=wc)
        assert got_n == nc
        ref = np.transpose(X, [t - 1 for t in tau])
        np.testing.assert_array_equal(_logical(buf, nc, wc), ref)


def test_transpose_permute_example():
    # Table 3: C = permute(A, [2, 1, 3]) swaps the first two modes
    X = synth.uniform((3, 4, 2), 32)
    mem, w = _mem(X, (1, 2, 3))
    buf, nc = oracle.transpose(mem, (3, 4, 2), w, (2, 1, 3))
    assert nc == (4, 3, 2)
    C = _logical(buf, nc, oracle.strides(nc))
    for i, j, k in itertools.product(range(3), range(4), range(2)):
        assert C[j, i, k] == X[i, j, k]


def test_transpose_then_inverse_is_identity():
    X = synth.uniform((2, 3, 4, 5, 2), 33)
    tau = (3, 5, 1, 2, 4)
    inv = tuple(int(x) + 1 for x in np.argsort(np.asarray(tau) - 1))
    mem, w = _mem(X, (1, 2, 3, 4, 5))
    buf, nc = oracle.transpose(mem, X.shape, w, tau)
    back, nb = oracle.transpose(buf, nc, oracle.strides(nc), inv)
    assert nb == X.shape
    np.testing.assert_array_equal(back, mem)


def test_transpose_rejects_non_permutation():
    X = synth.uniform((2, 3), 34)
    mem, w = _mem(X, (1, 2))
    with pytest.raises(ValueError):
        oracle.transpose(mem, (2, 3), w, (1, 1))


# ------------------------------------------------------------------- ttt ---

def _einsum_ttt(X, Y, q, phi, psi):
    pa, pb = X.ndim, Y.ndim
    r, s = pa - q, pb - q
    la = [None] * pa
    lb = [None] * pb
    it = iter(LETTERS)
    out = []
    for k in range(r):
        la[phi[k] - 1] = next(it)
        out.append(la[phi[k] - 1])
    for k in range(s):
        lb[psi[k] - 1] = next(it)
        out.append(lb[psi[k] - 1])
    for k in range(q):
        c = next(it)
        la[phi[r + k] - 1] = c
        lb[psi[s + k] - 1] = c
    return np.einsum(f"{''.join(la)},{''.join(lb)}->{''.join(out)}", X, Y)


def _random_ttt(g, q, r, s, emax=5):
    nj = [int(g.integers(1, emax + 1)) for _ in range(q)]
    na_free = [int(g.integers(1, emax + 1)) for _ in range(r)]
    nb_free = [int(g.integers(1, emax + 1)) for _ in range(s)]
    phi = [int(x) + 1 for x in g.permutation(q + r)]
    psi = [int(x) + 1 for x in g.permutation(q + s)]
    nA = [0] * (q + r)
    nB = [0] * (q + s)
    for k in range(r):
        nA[phi[k] - 1] = na_free[k]
    for k in range(s):
        nB[psi[k] - 1] = nb_free[k]
    for k in range(q):
        nA[phi[r + k] - 1] = nj[k]
        nB[psi[s + k] - 1] = nj[k]
    return tuple(nA), tuple(nB), phi, psi


@pytest.mark.parametrize("q,r,s", [(1, 2, 1), (2, 1, 2), (3, 1, 1), (2, 2, 0), (2, 0, 2),
                                   (0, 2, 2), (3, 0, 0), (1, 0, 1), (1, 3, 2)])
def test_ttt_matches_einsum(q, r, s, seed=0):
    g = synth.rng(40 + 7 * q + 3 * r + s + 100 * seed)
    for trial in range(4):
        nA, nB, phi, psi = _random_ttt(g, q, r, s)
        X = synth.uniform(nA, 41 + trial + 100 * seed)
        Y = synth.uniform(nB, 42 + trial + 100 * seed)
        pa, pb = synth.random_layout(len(nA), g), synth.random_layout(len(nB), g)
        ma, wa = _mem(X, pa)
        mb, wb = _mem(Y, pb)
        nc = oracle.ttt_shape(nA, nB, q, phi, psi)
        wc = oracle.strides(nc, synth.random_layout(len(nc), g)) if nc else ()
        buf, got_n = oracle.ttt(ma, nA, wa, phi, mb, nB, wb, psi, q, wC=wc)
        assert got_n == nc
        ref = _einsum_ttt(X, Y, q, phi, psi)
        assert np.allclose(_logical(buf, nc, wc), ref, rtol=1e-13, atol=1e-13)


def test_ttt_brute_force_tiny():
    # A 2x3x2, B 3x2x4: contract A's mode 2 with B's mode 1 and A's mode 3 with
    # B's mode 2; C(i, l) = sum_{j,k} A(i, j, k) B(j, k, l)
    X = synth.integers((2, 3, 2), 43)
    Y = synth.integers((3, 2, 4), 44)
    ma, wa = _mem(X, (3, 1, 2))
    mb, wb = _mem(Y, (2, 3, 1))
    buf, nc = oracle.ttt(ma, X.shape, wa, (1, 2, 3), mb, Y.shape, wb, (3, 1, 2), 2)
    assert nc == (2, 4)
    C = _logical(buf, nc, oracle.strides(nc))
    for i in range(2):
        for l in range(4):
            s = 0.0
            for j in range(3):
                for k in range(2):
                    s += X[i, j, k] * Y[j, k, l]
            assert C[i, l] == s


def test_ttt_reduces_to_ttv():
    # q = 1, r = p - 1, s = 0, phi = (1..m-1, m+1..p, m), psi = (1) is Eq. 24
    n = (4, 6, 3, 5)
    X = synth.uniform(n, 45)
    mem, w = _mem(X, (2, 4, 1, 3))
    for m in range(1, 5):
        b = synth.uniform((n[m - 1],), 46 + m)
        phi = [r for r in range(1, 5) if r != m] + [m]
        buf, nc = oracle.ttt(mem, n, w, phi, b, (n[m - 1],), (1,), (1,), 1)
        ref = np.tensordot(X, b, axes=([m - 1], [0]))
        assert np.allclose(buf.reshape(nc, order="F"), ref, rtol=1e-13)


def test_ttt_reduces_to_ttm_on_the_last_mode():
    # m = p, q = 1, r = p - 1, s = 1, phi = (1..p), psi = (1, 2) is Eq. 25
    n = (3, 4, 5)
    X = synth.uniform(n, 47)
    M = synth.uniform((7, 5), 48)
    mem, w = _mem(X, (1, 2, 3))
    buf, nc = oracle.ttt(mem, n, w, (1, 2, 3), M.reshape(-1), (7, 5), (5, 1), (1, 2), 1)
    assert nc == (3, 4, 7)
    ref = np.einsum("ijk,lk->ijl", X, M)
    assert np.allclose(buf.reshape(nc, order="F"), ref, rtol=1e-13)


def test_ttt_inner_and_outer_products():
    X = synth.uniform((3, 4, 2), 49)
    Y = synth.uniform((2, 3, 4), 50)
    ma, wa = _mem(X, (1, 2, 3))
    mb, wb = _mem(Y, (3, 1, 2))
    # inner product <A, B^tau> over all three modes (r = s = 0)
    buf, nc = oracle.ttt(ma, X.shape, wa, (1, 2, 3), mb, Y.shape, wb, (2, 3, 1), 3)
    assert nc == ()
    assert np.isclose(buf[0], np.sum(X * np.transpose(Y, (1, 2, 0))), rtol=1e-13)
    # outer product (q = 0): C = A o B with the modes of A first
    buf, nc = oracle.ttt(ma, X.shape, wa, (1, 2, 3), mb, Y.shape, wb, (1, 2, 3), 0)
    assert nc == (3, 4, 2, 2, 3, 4)
    assert np.allclose(buf.reshape(nc, order="F"), np.multiply.outer(X, Y), rtol=1e-15)


def test_ttt_worked_example_shapes():
    # Sec. 5.2 example: A {3,4,2} and B {5,4,3,6} share the extents 3 and 4;
    # contracting them (phi = (3,1,2), psi = (1,4,3,2)) leaves C {2,5,6}
    nA, nB = (3, 4, 2), (5, 4, 3, 6)
    X, Y = synth.uniform(nA, 51), synth.uniform(nB, 52)
    ma, wa = _mem(X, (1, 2, 3))
    mb, wb = _mem(Y, (1, 2, 3, 4))
    buf, nc = oracle.ttt(ma, nA, wa, (3, 1, 2), mb, nB, wb, (1, 4, 3, 2), 2)
    assert nc == (2, 5, 6)
    ref = np.einsum("ijk,ljim->klm", X, Y)
    assert np.allclose(buf.reshape(nc, order="F"), ref, rtol=1e-13)


def test_ttt_rejects_mismatched_contraction():
    X, Y = synth.uniform((3, 4), 53), synth.uniform((5, 4), 54)
    ma, wa = _mem(X, (1, 2))
    mb, wb = _mem(Y, (1, 2))
    with pytest.raises(ValueError):
        oracle.ttt(ma, (3, 4), wa, (2, 1), mb, (5, 4), wb, (2, 1), 1)   # 3 vs 4


def test_ttt_integer_inputs_exact():
    g = synth.rng(55)
    nA, nB, phi, psi = _random_ttt(g, 2, 2, 1, emax=6)
    X, Y = synth.integers(nA, 56), synth.integers(nB, 57)
    ma, wa = _mem(X, synth.random_layout(len(nA), g))
    mb, wb = _mem(Y, synth.random_layout(len(nB), g))
    buf, nc = oracle.ttt(ma, nA, wa, phi, mb, nB, wb, psi, 2)
    np.testing.assert_array_equal(buf.reshape(nc, order="F"), _einsum_ttt(X, Y, 2, phi, psi))


def test_ttt_times_tensor_example_shapes():
    # Sec. 5.2 member-function example: A {3,4,2,6} times C {2,3,4}, contracting
    # A's modes 2, 3 with C's modes 3, 1, leaves A's modes 1, 4 then C's mode 2:
    # in (q, phi, psi) form q = 2, phi = (1,4,2,3), psi = (2,3,1) -> {3,6,3}
    nA, nC = (3, 4, 2, 6), (2, 3, 4)
    X, Y = synth.uniform(nA, 58), synth.uniform(nC, 59)
    ma, wa = _mem(X, (1, 2, 3, 4))
    mc, wc = _mem(Y, (1, 2, 3))
    buf, nd = oracle.ttt(ma, nA, wa, (1, 4, 2, 3), mc, nC, wc, (2, 3, 1), 2)
    assert nd == (3, 6, 3)
    ref = np.einsum("ijkl,kmj->ilm", X, Y)
    assert np.allclose(buf.reshape(nd, order="F"), ref, rtol=1e-13)

"""Pins for the oracle's times_vectors, times_matrices and higher-order power
method (Sec. 5.2 Table 3 and the HOPM listing) against closed forms, numpy
einsum / SVD, and the special cases the definitions fix."""
import numpy as np
import pytest

import oracle
import synth


def _mem(X, pi):
    return synth.to_memory(X, pi), oracle.strides(X.shape, pi)


def test_ttvs_matches_einsum_any_layout():
    g = synth.rng(11)
    n = (5, 4, 6, 3)
    X = synth.uniform(n, 12)
    vs = [synth.uniform((x,), 13 + i) for i, x in enumerate(n)]
    for modes in ([1, 2, 4], [3], [4, 2], [2, 3, 4]):
        pi = synth.random_layout(4, g)
        mem, w = _mem(X, pi)
        got, rest = oracle.ttvs(mem, n, w, modes, [vs[m - 1] for m in modes])
        letters = "abcd"
        keep = "".join(letters[r] for r in range(4) if r + 1 not in modes)
        ref = np.einsum(f"abcd,{','.join(letters[m - 1] for m in modes)}->{keep}", X,
                        *[vs[m - 1] for m in modes])
        assert rest == tuple(n[r] for r in range(4) if r + 1 not in modes)
        got_l = got.reshape(rest, order="F") if rest else got[:1]
        assert np.allclose(got_l, ref, rtol=1e-13, atol=1e-13)


def test_ttvs_leaves_at_least_one_mode():
    # ttv needs order >= 2 (Eq. 24), so a sequence keeps at least one mode
    X = synth.uniform((3, 4), 18)
    mem, w = _mem(X, (1, 2))
    with pytest.raises(ValueError):
        oracle.ttvs(mem, (3, 4), w, [1, 2], [np.ones(3), np.ones(4)])


def test_ttvs_paper_example_shapes():
    # Sec. 5.2: A {3,4,2,6} with vectors along modes {1,2,4} leaves mode 3 (2)
    X = synth.uniform((3, 4, 2, 6), 14)
    mem, w = _mem(X, (1, 2, 3, 4))
    vs = [synth.uniform((3,), 15), synth.uniform((4,), 16), synth.uniform((6,), 17)]
    out, rest = oracle.ttvs(mem, (3, 4, 2, 6), w, [1, 2, 4], vs)
    assert rest == (2,)


def test_ttvs_rank_one_closed_form():
    a, b, c = synth.uniform((4,), 20), synth.uniform((5,), 21), synth.uniform((3,), 22)
    X = 2.5 * np.einsum("i,j,k->ijk", a, b, c)
    u, v = synth.uniform((4,), 23), synth.uniform((3,), 24)
    mem, w = _mem(X, (2, 3, 1))
    out, rest = oracle.ttvs(mem, X.shape, w, [1, 3], [u, v])
    assert np.allclose(out, 2.5 * (a @ u) * (c @ v) * b, rtol=1e-13)


def test_ttms_matches_einsum_and_tucker_shape():
    n = (6, 5, 4)
    X = synth.uniform(n, 30)
    U = [synth.uniform((3, 6), 31), synth.uniform((2, 5), 32), synth.uniform((2, 4), 33)]
    mem, w = _mem(X, (3, 1, 2))
    out, rest = oracle.ttms(mem, n, w, [1, 2, 3], U)
    assert rest == (3, 2, 2)
    ref = np.einsum("abc,ia,jb,kc->ijk", X, *U)
    assert np.allclose(out.reshape(rest, order="F"), ref, rtol=1e-13, atol=1e-14)


def test_ttms_order_independent_on_integers():
    n = (4, 3, 5)
    X = synth.integers(n, 34)
    U = [synth.integers((2, 4), 35), synth.integers((3, 5), 36)]
    mem, w = _mem(X, (1, 2, 3))
    a, _ = oracle.ttms(mem, n, w, [1, 3], U)
    b, _ = oracle.ttms(mem, n, w, [3, 1], U[::-1])
    np.testing.assert_array_equal(a, b)


def test_hopm_rank_one_converges_in_one_sweep():
    # A = sigma a o b o c with unit a, b, c: the first sweep returns u_r = +-a_r
    # and, after its last step, lambda_p = sigma exactly (up to rounding)
    g = synth.rng(40)
    vs = [g.standard_normal(x) for x in (5, 4, 6)]
    vs = [v / np.linalg.norm(v) for v in vs]
    sigma = 3.75
    X = sigma * np.einsum("i,j,k->ijk", *vs)
    mem, w = _mem(X, (3, 1, 2))
    u0 = [np.ones(x) for x in X.shape]
    u, lam = oracle.hopm(mem, X.shape, w, u0, 1)
    assert abs(lam[-1] - sigma) <= 1e-13 * sigma
    for ur, vr in zip(u, vs):
        assert abs(abs(ur @ vr) - 1.0) <= 1e-13


def test_hopm_on_a_matrix_is_power_iteration():
    # p = 2: u1 <- A u2, u2 <- A^T u1 converges to the top singular pair
    A = synth.uniform((7, 5), 41)
    mem, w = _mem(A, (1, 2))
    u, lam = oracle.hopm(mem, A.shape, w, [np.ones(7), np.ones(5)], 60)
    s = np.linalg.svd(A, compute_uv=False)
    assert abs(lam[0] - s[0]) <= 1e-10 * s[0]
    assert abs(lam[1] - s[0]) <= 1e-10 * s[0]


def test_hopm_lambda_never_decreases_within_a_sweep():
    X = synth.uniform((4, 5, 3, 3), 42)
    mem, w = _mem(X, (1, 2, 3, 4))
    u, lam_prev = oracle.hopm(mem, X.shape, w, [np.ones(x) for x in X.shape], 1)
    for k in range(2, 6):
        _, lam = oracle.hopm(mem, X.shape, w, [np.ones(x) for x in X.shape], k)
        assert lam[-1] >= lam_prev[-1] - 1e-12
        lam_prev = lam

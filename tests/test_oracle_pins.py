"""Pins the FP64 oracle to things other than itself (CPU only).

Each check compares the oracle with a value the paper prints (fixtures under
tests/golden/), a closed form the paper states, numpy's own memory layouts and
library routines (tensordot, matmul, norm), a stated special case, or brute
force over tiny inputs.  Together they are chosen so that a dropped term, a
wrong index, a transposed operand or a wrong sign in the oracle fails at least
one check (tests/test_oracle_mutations.py plants such mistakes and confirms).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import ints, read_golden


def logical_to_mem(X, pi):
    return synth.to_memory(X, pi)


def mem_to_logical(mem, n, pi):
    return synth.from_memory(mem, n, pi)


# ----------------------------------------------------------------- layout ---

def test_strides_printed_examples():
    rows = read_golden("strides_examples.txt")
    assert len(rows) == 3
    for row in rows:
        n, pi, w, _ = [c.strip() for c in row.split("|")]
        assert oracle.strides(ints(n), ints(pi)) == ints(w)


def test_strides_default_is_first_order():
    assert oracle.strides((4, 2, 3)) == (1, 4, 8)


@pytest.mark.parametrize("seed", range(6))
def test_strides_closed_forms_first_and_last_order(seed):
    # Sec. 3.1 Eq. 15: w_F = (1, n1, n1 n2, ...); Eq. 16: w_L = (n2..np, ..., np, 1)
    g = synth.rng(seed)
    p = int(g.integers(1, 8))
    n = tuple(int(x) for x in g.integers(1, 9, size=p))
    wF = tuple(int(np.prod(n[:r])) for r in range(p))
    wL = tuple(int(np.prod(n[r + 1:])) for r in range(p))
    assert oracle.strides(n, synth.first_order(p)) == wF
    assert oracle.strides(n, synth.last_order(p)) == wL


def test_strides_monotone_in_layout_order():
    # Sec. 3.1: 1 <= w_{pi_q} <= w_{pi_r} for q < r
    g = synth.rng(7)
    for _ in range(50):
        p = int(g.integers(1, 7))
        n = tuple(int(x) for x in g.integers(1, 6, size=p))
        pi = synth.random_layout(p, g)
        w = oracle.strides(n, pi)
        seq = [w[r - 1] for r in pi]
        assert seq[0] == 1 and all(a <= b for a, b in zip(seq, seq[1:]))


def test_strides_reject_non_permutation():
    with pytest.raises(ValueError):
        oracle.strides((2, 3, 4), (1, 1, 3))
    with pytest.raises(ValueError):
        oracle.strides((2, 3), (0, 1))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_layout_function_bijective_for_every_layout(p):
    # brute force: for every pi in Pi_p the memory indices of all multi-indices
    # form exactly the memory index set {0..N-1} (Sec. 3.1, Eq. 11)
    g = synth.rng(100 + p)
    n = tuple(int(x) for x in g.integers(1, 5, size=p))
    N = int(np.prod(n))
    for pi in synth.all_layouts(p):
        w = oracle.strides(n, pi)
        offs = sorted(oracle.lam(w, i) for i in itertools.product(*[range(x) for x in n]))
        assert offs == list(range(N))


@pytest.mark.parametrize("seed", range(8))
def test_layout_function_matches_numpy_storage(seed):
    # numpy's transpose+ravel storage of a logical array in layout pi puts
    # X[i] at the memory index lambda(w(pi), i) (Eqs. 14 and 17)
    g = synth.rng(200 + seed)
    p = int(g.integers(1, 6))
    n = tuple(int(x) for x in g.integers(1, 6, size=p))
    pi = synth.random_layout(p, g)
    X = np.arange(int(np.prod(n)), dtype=np.float64).reshape(n) * 3 + 1
    mem = logical_to_mem(X, pi)
    w = oracle.strides(n, pi)
    for i in itertools.product(*[range(x) for x in n]):
        assert mem[oracle.lam(w, i)] == X[i]


def test_layout_function_offsets():
    # Sec. 3.2 Example: B(shape {4,2,3}, offset {1,-1,0}, layout {3,2,1}):
    # the first element (i = o) has memory index 0; lambda is shift-invariant
    n, o, pi = (4, 2, 3), (1, -1, 0), (3, 2, 1)
    w = oracle.strides(n, pi)
    assert oracle.lam(w, o, o) == 0
    for i0 in itertools.product(range(4), range(2), range(3)):
        i = tuple(a + b for a, b in zip(i0, o))
        assert oracle.lam(w, i, o) == oracle.lam(w, i0)


def test_matlab_print_example_last_order():
    # Sec. 3.4: a last-order (3,4,2) tensor holding its memory indices
    rows = read_golden("matlab_print_last_order_3x4x2.txt")
    w = oracle.strides((3, 4, 2), synth.last_order(3))
    seen = 0
    for row in rows:
        s, r, vals = [c.strip() for c in row.split("|")]
        for col, v in enumerate(int(x) for x in vals.split()):
            assert oracle.lam(w, (int(r), col, int(s))) == v
            seen += 1
    assert seen == 24


def test_view_example():
    rows = read_golden("view_example_4x2x3.txt")
    n, f, t, l, nv_expect = [ints(c) for c in rows[0].split("|")]
    w = oracle.strides(n)
    nv, wv, gamma = oracle.view(n, w, f, t, l)
    assert nv == nv_expect
    for row in rows[1:]:
        iv, ia = [ints(c) for c in row.split("->")]
        # Eq. 19: lambda'(w', i', o) = gamma + lambda(w'', i', o)
        assert gamma + oracle.lam(wv, iv) == oracle.lam(w, ia)


def test_view_with_offsets_and_bounds():
    n, o = (4, 2, 3), (1, -1, 0)
    w = oracle.strides(n, (3, 2, 1))
    f, t, l = (2, -1, 0), (2, 1, 1), (4, 0, 2)
    nv, wv, gamma = oracle.view(n, w, f, t, l, o)
    assert nv == (2, 2, 3)
    assert gamma == oracle.lam(w, f, o)
    assert wv == tuple(a * b for a, b in zip(w, t))
    with pytest.raises(ValueError):
        oracle.view(n, w, (0, 0, 0), (1, 1, 1), (4, 1, 2))      # l beyond n with o=0
    with pytest.raises(ValueError):
        oracle.view(n, w, (0, 0, 0), (0, 1, 1), (3, 1, 2))      # zero step


def test_stride_iterator_fiber_example():
    (row,) = read_golden("stride_iterator_fiber.txt")
    n, pi, fixed, mem = [c.strip() for c in row.split("|")]
    n, pi, mem = ints(n), ints(pi), ints(mem)
    w = oracle.strides(n, pi)
    parts = fixed.split(",")
    run = parts.index("*")
    got = []
    for i in range(n[run]):
        idx = [int(x) if x != "*" else i for x in parts]
        got.append(oracle.lam(w, idx))
    assert tuple(got) == mem


# -------------------------------------------------------------------- ttv ---

def _rand_case(g, pmin=2, pmax=5, emax=6):
    p = int(g.integers(pmin, pmax + 1))
    n = tuple(int(x) for x in g.integers(1, emax + 1, size=p))
    return p, n


def _oracle_ttv_logical(X, q, b, pi_a, pi_c=None, accumulate=False, C0=None):
    n = X.shape
    p = len(n)
    wA = oracle.strides(n, pi_a)
    nout = tuple(x for r, x in enumerate(n) if r != q - 1)
    if pi_c is None:
        pi_c = synth.first_order(p - 1)
    wC = oracle.strides(nout, pi_c)
    C = None if C0 is None else logical_to_mem(C0, pi_c)
    Cm = oracle.ttv(logical_to_mem(X, pi_a), n, wA, q, b, C=C, wC=wC, accumulate=accumulate)
    return mem_to_logical(Cm, nout, pi_c)


@pytest.mark.parametrize("seed", range(12))
def test_ttv_matches_tensordot(seed):
    g = synth.rng(300 + seed)
    p, n = _rand_case(g)
    q = int(g.integers(1, p + 1))
    X = synth.uniform(n, 1000 + seed)
    b = synth.uniform((n[q - 1],), 2000 + seed)
    pi_a = synth.random_layout(p, g)
    pi_c = synth.random_layout(p - 1, g)
    got = _oracle_ttv_logical(X, q, b, pi_a, pi_c)
    ref = np.tensordot(X, b, axes=([q - 1], [0]))
    # FP64 bound for a length-n_q dot product: n_q * eps * sum |a_k b_k|
    bound = n[q - 1] * 2.3e-16 * np.tensordot(np.abs(X), np.abs(b), axes=([q - 1], [0]))
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


@pytest.mark.parametrize("seed", range(6))
def test_ttv_integer_inputs_exact(seed):
    g = synth.rng(400 + seed)
    p, n = _rand_case(g, emax=8)
    q = int(g.integers(1, p + 1))
    X = synth.integers(n, 3000 + seed)
    b = synth.integers((n[q - 1],), 4000 + seed)
    got = _oracle_ttv_logical(X, q, b, synth.random_layout(p, g))
    np.testing.assert_array_equal(got, np.tensordot(X, b, axes=([q - 1], [0])))


def test_ttv_unit_vector_gives_slice():
    g = synth.rng(5)
    n = (5, 4, 3, 2)
    X = synth.uniform(n, 77)
    for q in range(1, 5):
        for k in range(n[q - 1]):
            e = np.zeros(n[q - 1])
            e[k] = 1.0
            got = _oracle_ttv_logical(X, q, e, synth.random_layout(4, g))
            np.testing.assert_array_equal(got, np.take(X, k, axis=q - 1))


def test_ttv_ones_gives_mode_sums():
    n = (3, 5, 4)
    X = synth.integers(n, 78)
    for q in (1, 2, 3):
        got = _oracle_ttv_logical(X, q, np.ones(n[q - 1]), synth.last_order(3))
        np.testing.assert_array_equal(got, X.sum(axis=q - 1))


def test_ttv_p2_is_vector_matrix_product():
    # Sec. 5.2 after Eq. 24: for p = 2 and m = 1, ttv is a vector-matrix product
    A = synth.integers((6, 7), 79)
    b = synth.integers((6,), 80)
    got = _oracle_ttv_logical(A, 1, b, (1, 2))
    np.testing.assert_array_equal(got, b @ A)
    b2 = synth.integers((7,), 81)
    np.testing.assert_array_equal(_oracle_ttv_logical(A, 2, b2, (2, 1)), A @ b2)


def test_ttv_brute_force_tiny():
    g = synth.rng(82)
    for _ in range(10):
        p, n = _rand_case(g, pmax=4, emax=3)
        q = int(g.integers(1, p + 1))
        X = synth.uniform(n, int(g.integers(1 << 30)))
        b = synth.uniform((n[q - 1],), int(g.integers(1 << 30)))
        got = _oracle_ttv_logical(X, q, b, synth.random_layout(p, g))
        nout = [x for r, x in enumerate(n) if r != q - 1]
        for iout in itertools.product(*[range(x) for x in nout]):
            s = 0.0
            for k in range(n[q - 1]):
                full = list(iout)
                full.insert(q - 1, k)
                s += X[tuple(full)] * b[k]
            assert got[iout] == s


def test_ttv_layout_invariance_bit_exact():
    # equality of tensors is layout independent (Sec. 3.2); the oracle's
    # result per multi-index must not depend on pi_A or pi_C
    n = (3, 4, 2, 5)
    X = synth.uniform(n, 83)
    for q in range(1, 5):
        b = synth.uniform((n[q - 1],), 84 + q)
        base = _oracle_ttv_logical(X, q, b, synth.first_order(4))
        for pi in synth.all_layouts(4)[::3]:
            pic = tuple(r for r in synth.last_order(3))
            np.testing.assert_array_equal(_oracle_ttv_logical(X, q, b, pi, pic), base)


def test_ttv_accumulate_adds_to_existing_output():
    n = (4, 3, 5)
    X = synth.integers(n, 90)
    b = synth.integers((3,), 91)
    C0 = synth.integers((4, 5), 92)
    got = _oracle_ttv_logical(X, 2, b, (2, 3, 1), (2, 1), accumulate=True, C0=C0)
    np.testing.assert_array_equal(got, C0 + np.tensordot(X, b, axes=([1], [0])))


def test_ttv_at_matches_full():
    g = synth.rng(93)
    n = (7, 5, 6)
    X = synth.uniform(n, 94)
    pi = (3, 1, 2)
    mem = logical_to_mem(X, pi)
    w = oracle.strides(n, pi)
    for q in (1, 2, 3):
        b = synth.uniform((n[q - 1],), 95 + q)
        nout = tuple(x for r, x in enumerate(n) if r != q - 1)
        full = mem_to_logical(oracle.ttv(mem, n, w, q, b), nout, synth.first_order(2))
        idx = np.stack([g.integers(0, x, size=20) for x in nout], axis=1)
        pts = oracle.ttv_at(mem, n, w, q, b, idx)
        np.testing.assert_array_equal(pts, full[tuple(idx.T)])


def test_ttv_output_shape_examples():
    for row in read_golden("output_shapes.txt"):
        op, na, q, nb, nc = [c.strip() for c in row.split("|")]
        if op != "ttv":
            continue
        na, q, nc = ints(na), int(q), ints(nc)
        X = synth.uniform(na, 96)
        b = synth.uniform((ints(nb)[0],), 97)
        got = _oracle_ttv_logical(X, q, b, synth.first_order(len(na)))
        assert got.shape == nc


# -------------------------------------------------------------------- ttm ---

def _oracle_ttm_logical(X, q, B, pi_a, pi_c=None, accumulate=False, C0=None, ldb_col=1):
    n = X.shape
    p = len(n)
    J = B.shape[0]
    wA = oracle.strides(n, pi_a)
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    if pi_c is None:
        pi_c = pi_a
    wC = oracle.strides(nout, pi_c)
    C = None if C0 is None else logical_to_mem(C0, pi_c)
    if ldb_col == 1:
        Bbuf, ldr, ldc = np.ascontiguousarray(B).reshape(-1), B.shape[1], 1
    else:  # B stored column-major
        Bbuf, ldr, ldc = np.ascontiguousarray(B.T).reshape(-1), 1, B.shape[0]
    Cm = oracle.ttm(logical_to_mem(X, pi_a), n, wA, q, Bbuf, J, ldr, ldc, C=C, wC=wC,
                    accumulate=accumulate)
    return mem_to_logical(Cm, nout, pi_c)


def _tensordot_ttm(X, B, q):
    return np.moveaxis(np.tensordot(X, B, axes=([q - 1], [1])), -1, q - 1)


def test_ttm_identity_returns_input():
    n = (5, 3, 4, 2)
    X = synth.uniform(n, 100)
    g = synth.rng(101)
    for q in range(1, 5):
        I = np.eye(n[q - 1])
        got = _oracle_ttm_logical(X, q, I, synth.random_layout(4, g), synth.random_layout(4, g))
        np.testing.assert_array_equal(got, X)


def test_ttm_permutation_matrix_permutes_slices():
    n = (4, 6, 3)
    X = synth.uniform(n, 102)
    g = synth.rng(103)
    for q in (1, 2, 3):
        perm = g.permutation(n[q - 1])
        P = np.eye(n[q - 1])[perm]           # P(j, k) = 1 iff k == perm[j]
        got = _oracle_ttm_logical(X, q, P, synth.last_order(3))
        np.testing.assert_array_equal(got, np.take(X, perm, axis=q - 1))


def test_ttm_single_row_equals_ttv():
    # Sec. 5.2 after Eq. 25: with n' = 1 the tensor-matrix product is ttv
    n = (3, 5, 4)
    X = synth.uniform(n, 104)
    for q in (1, 2, 3):
        b = synth.uniform((n[q - 1],), 105 + q)
        got = _oracle_ttm_logical(X, q, b[None, :], synth.first_order(3))
        np.testing.assert_array_equal(np.squeeze(got, axis=q - 1),
                                      _oracle_ttv_logical(X, q, b, synth.first_order(3)))


def test_ttm_p2_is_matrix_product():
    # Sec. 5.2 after Eq. 25: for p = 2 ttm is a matrix-matrix product
    A = synth.integers((5, 7), 110)
    B1 = synth.integers((3, 5), 111)
    B2 = synth.integers((4, 7), 112)
    np.testing.assert_array_equal(_oracle_ttm_logical(A, 1, B1, (1, 2)), B1 @ A)
    np.testing.assert_array_equal(_oracle_ttm_logical(A, 2, B2, (2, 1)), A @ B2.T)
    # random data against a textbook triple loop
    A = synth.uniform((4, 6), 113)
    B = synth.uniform((3, 4), 114)
    got = _oracle_ttm_logical(A, 1, B, (2, 1), ldb_col=3)
    for j in range(3):
        for c in range(6):
            s = 0.0
            for k in range(4):
                s += B[j, k] * A[k, c]
            assert got[j, c] == s


@pytest.mark.parametrize("seed", range(10))
def test_ttm_matches_tensordot(seed):
    g = synth.rng(500 + seed)
    p, n = _rand_case(g)
    q = int(g.integers(1, p + 1))
    J = int(g.integers(1, 6))
    X = synth.uniform(n, 5000 + seed)
    B = synth.uniform((J, n[q - 1]), 6000 + seed)
    got = _oracle_ttm_logical(X, q, B, synth.random_layout(p, g), synth.random_layout(p, g))
    ref = _tensordot_ttm(X, B, q)
    bound = n[q - 1] * 2.3e-16 * _tensordot_ttm(np.abs(X), np.abs(B), q)
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


def test_ttm_distinct_modes_commute():
    n = (4, 5, 3)
    X = synth.integers(n, 120)
    U = synth.integers((2, 5), 121)
    V = synth.integers((6, 3), 122)
    lhs = _oracle_ttm_logical(_oracle_ttm_logical(X, 2, U, (1, 2, 3)), 3, V, (3, 1, 2))
    rhs = _oracle_ttm_logical(_oracle_ttm_logical(X, 3, V, (2, 3, 1)), 2, U, (1, 2, 3))
    np.testing.assert_array_equal(lhs, rhs)   # integer data: exact
    Xr = synth.uniform(n, 123)
    Ur, Vr = synth.uniform((2, 5), 124), synth.uniform((6, 3), 125)
    a = _oracle_ttm_logical(_oracle_ttm_logical(Xr, 2, Ur, (1, 2, 3)), 3, Vr, (1, 2, 3))
    b = _oracle_ttm_logical(_oracle_ttm_logical(Xr, 3, Vr, (1, 2, 3)), 2, Ur, (1, 2, 3))
    assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(a)


def test_ttm_brute_force_tiny():
    g = synth.rng(126)
    for _ in range(8):
        p, n = _rand_case(g, pmax=4, emax=3)
        q = int(g.integers(1, p + 1))
        J = int(g.integers(1, 4))
        X = synth.uniform(n, int(g.integers(1 << 30)))
        B = synth.uniform((J, n[q - 1]), int(g.integers(1 << 30)))
        got = _oracle_ttm_logical(X, q, B, synth.random_layout(p, g))
        nout = [J if r == q - 1 else x for r, x in enumerate(n)]
        for iout in itertools.product(*[range(x) for x in nout]):
            s = 0.0
            for k in range(n[q - 1]):
                full = list(iout)
                full[q - 1] = k
                s += X[tuple(full)] * B[iout[q - 1], k]
            assert got[iout] == s


def test_ttm_accumulate_and_at():
    n = (3, 4, 5)
    X = synth.integers(n, 127)
    B = synth.integers((2, 4), 128)
    C0 = synth.integers((3, 2, 5), 129)
    got = _oracle_ttm_logical(X, 2, B, (1, 2, 3), (3, 1, 2), accumulate=True, C0=C0)
    np.testing.assert_array_equal(got, C0 + _tensordot_ttm(X, B, 2))
    mem = logical_to_mem(X, (2, 3, 1))
    w = oracle.strides(n, (2, 3, 1))
    idx = np.array([[0, 0, 0], [2, 1, 4], [1, 0, 3]])
    pts = oracle.ttm_at(mem, n, w, 2, B.reshape(-1), 4, 1, idx)
    ref = _tensordot_ttm(X, B, 2)
    np.testing.assert_array_equal(pts, ref[tuple(idx.T)])


def test_ttm_output_shape_example():
    for row in read_golden("output_shapes.txt"):
        op, na, q, nb, nc = [c.strip() for c in row.split("|")]
        if op != "ttm":
            continue
        X = synth.uniform(ints(na), 130)
        B = synth.uniform(ints(nb), 131)
        assert _oracle_ttm_logical(X, int(q), B, synth.first_order(3)).shape == ints(nc)


# ------------------------------------------------------------- entrywise ---

@pytest.mark.parametrize("op", [oracle.OP_ADD, oracle.OP_SUB, oracle.OP_MUL, oracle.OP_DIV,
                                oracle.OP_COPY, oracle.OP_SCALE])
def test_entrywise_mixed_layouts_against_numpy(op):
    g = synth.rng(140 + op)
    n = (3, 4, 2, 5)
    X = synth.uniform(n, 141)
    Y = synth.uniform(n, 142) + 2.0
    pa, pb, pc = (synth.random_layout(4, g) for _ in range(3))
    wA, wB, wC = (oracle.strides(n, pi) for pi in (pa, pb, pc))
    Cm = oracle.entrywise(op, n, logical_to_mem(X, pa), wA, logical_to_mem(Y, pb), wB,
                          alpha=-1.5, wC=wC)
    got = mem_to_logical(Cm, n, pc)
    ref = {oracle.OP_ADD: X + Y, oracle.OP_SUB: X - Y, oracle.OP_MUL: X * Y,
           oracle.OP_DIV: X / Y, oracle.OP_COPY: X, oracle.OP_SCALE: -1.5 * X}[op]
    np.testing.assert_array_equal(got, ref)


def test_entrywise_first_plus_last_order_small_case():
    case = synth.small_case()
    n = case.n
    mF = logical_to_mem(case.X, synth.first_order(3))
    mL = logical_to_mem(case.X, synth.last_order(3))
    Cm = oracle.entrywise(oracle.OP_ADD, n, mF, oracle.strides(n), mL,
                          oracle.strides(n, synth.last_order(3)))
    np.testing.assert_array_equal(mem_to_logical(Cm, n, synth.first_order(3)), 2 * case.X)


# ------------------------------------------------------------------ norms ---

def test_norm_against_numpy_and_closed_forms():
    n = (6, 5, 4)
    X = synth.uniform(n, 150)
    pi = (2, 3, 1)
    mem = logical_to_mem(X, pi)
    w = oracle.strides(n, pi)
    assert abs(oracle.norm(mem, n, w) - np.linalg.norm(X.ravel())) <= 1e-14 * np.linalg.norm(X)
    e = np.zeros(n)
    e[2, 1, 3] = 1.0
    assert oracle.norm(logical_to_mem(e, pi), n, w) == 1.0
    c = np.full(n, -3.0)
    assert abs(oracle.norm(logical_to_mem(c, pi), n, w) - 3.0 * math.sqrt(120)) < 1e-13


def test_rel_error_closed_form():
    n = (4, 3, 5)
    R = synth.uniform(n, 151)
    for eps in (1e-3, -2e-7, 0.0):
        Xm = logical_to_mem(R * (1 + eps), (3, 2, 1))
        got = oracle.rel_error(Xm, oracle.strides(n, (3, 2, 1)), logical_to_mem(R, (1, 2, 3)),
                               oracle.strides(n), n)
        assert abs(got - abs(eps)) <= 1e-15 + 1e-9 * abs(eps)

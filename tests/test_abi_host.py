"""Host-only checks of the C-ABI library (no GPU): every symbol declared in
include/tlgb.h is exported, argument validation returns the documented codes,
and the planner's collapsed iteration space enumerates exactly the element
pairs of the uncollapsed description."""
import itertools
import json
import os
import re

import numpy as np
import pytest

import oracle
import synth
from conftest import ROOT

FAKE = 1 << 20          # a non-null, 16-byte aligned fake device address


def declared_functions():
    with open(os.path.join(ROOT, "include", "tlgb.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for must in ("tl_ttv", "tl_ttm", "tl_entrywise", "tl_batch_submit", "tl_poll",
                 "tl_norm", "tl_strerror", "tl_ctx_create"):
        assert must in names


def test_library_exports_every_declared_symbol(tl):
    for name in declared_functions():
        assert hasattr(tl._lib, name), f"{name} not exported by libtlgb.so"


def test_binding_constants_match_the_header(tl):
    # the binding restates a few of tlgb.h's macros; they must not drift apart
    with open(os.path.join(ROOT, "include", "tlgb.h")) as fh:
        src = fh.read()
    m = re.search(r"#define\s+TL_TTV_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", src)
    assert m, "TL_TTV_NOALLOC_SCRATCH_BYTES not found in tlgb.h"
    assert tl.TL_TTV_NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))
    for name in ("TL_OK", "TL_EINVAL", "TL_EUNSUPPORTED", "TL_ENOMEM", "TL_ECUDA", "TL_ETIMEOUT",
                 "TL_ECANCELED", "TL_EBOUNDS",
                 "TL_P_F64", "TL_P_F32", "TL_P_TF32", "TL_P_BF16", "TL_P_BF16X3",
                 "TL_OP_TTV", "TL_OP_TTM", "TL_OP_ENTRYWISE"):
        m = re.search(r"#define\s+%s\s+(-?\d+)" % name, src)
        if m and hasattr(tl, name):
            assert getattr(tl, name) == int(m.group(1)), name


def test_strerror_and_version(tl):
    assert tl.tl_version() >= 100
    assert tl.tl_strerror(tl.TL_EINVAL) == "invalid argument"
    assert tl.tl_strerror(12345) == "unknown error"


def _desc(tl, n, pi=None, w=None, dtype="f32", addr=FAKE):
    return tl.Desc(addr, n, pi, w, dtype=dtype)


def _plan(tl, op, A, C, q=0, B=None, J=0, prec=0, eop=0):
    rc, js = tl.tl_plan_describe(op, A, B, q, J, prec, eop, C)
    return rc, (json.loads(js) if rc == 0 else None)


def test_plan_config2_kernels(tl):
    n = (128,) * 4
    for pi, q, kern, dims in [
        ((1, 2, 3, 4), 1, "ttv_row", [[128 ** 3, 128, 1]]),
        ((1, 2, 3, 4), 2, "ttv_col", [[128, 1, 1], [128 ** 2, 128 ** 2, 128]]),
        ((1, 2, 3, 4), 4, "ttv_col", [[128 ** 3, 1, 1]]),
        ((4, 3, 2, 1), 4, "ttv_row", [[128 ** 3, 128, 1]]),
    ]:
        A = _desc(tl, n, pi)
        nout = tuple(x for r, x in enumerate(n) if r != q - 1)
        pic = tuple(r for r in pi if r != q)
        pic = tuple(sorted(pic).index(r) + 1 for r in pic)   # induced layout
        C = _desc(tl, nout, pic, addr=FAKE * 2 ** 12)
        rc, P = _plan(tl, tl.TL_OP_TTV, A, C, q=q)
        assert rc == 0
        assert P["kernel"] == kern
        assert P["dims"] == dims
        assert P["splits"] == 1
        assert P["vec"] == 4


def _enumerate_pairs(space, nops):
    """All per-operand offset tuples of a collapsed space."""
    out = set()
    exts = [d[0] for d in space]
    for idx in itertools.product(*[range(e) for e in exts]):
        out.add(tuple(sum(i * d[1 + o] for i, d in zip(idx, space)) for o in range(nops)))
    return out


@pytest.mark.parametrize("seed", range(20))
def test_collapse_preserves_element_pairs_ttv(tl, seed):
    g = synth.rng(700 + seed)
    p = int(g.integers(2, 6))
    n = tuple(int(x) for x in g.integers(1, 5, size=p))
    q = int(g.integers(1, p + 1))
    pa = synth.random_layout(p, g)
    nout = tuple(x for r, x in enumerate(n) if r != q - 1)
    pc = synth.random_layout(p - 1, g)
    wA, wC = oracle.strides(n, pa), oracle.strides(nout, pc)
    rc, P = _plan(tl, tl.TL_OP_TTV, _desc(tl, n, pa), _desc(tl, nout, pc, addr=FAKE * 4096), q=q)
    assert rc == 0
    assert P["nq"] == n[q - 1] and P["saq"] == wA[q - 1]
    expect = set()
    for i in itertools.product(*[range(x) for x in nout]):
        full = list(i)
        full.insert(q - 1, 0)
        expect.add((oracle.lam(wA, full), oracle.lam(wC, i)))
    assert _enumerate_pairs(P["dims"], 2) == expect
    assert P["nout"] == int(np.prod(nout))


@pytest.mark.parametrize("seed", range(20))
def test_collapse_preserves_element_triples_entrywise(tl, seed):
    g = synth.rng(800 + seed)
    p = int(g.integers(1, 6))
    n = tuple(int(x) for x in g.integers(1, 5, size=p))
    pa, pb, pc = (synth.random_layout(p, g) for _ in range(3))
    w = [oracle.strides(n, pi) for pi in (pa, pb, pc)]
    rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, n, pa), _desc(tl, n, pc, addr=FAKE * 4096),
                  B=_desc(tl, n, pb, addr=FAKE * 8192), eop=tl.TL_ADD)
    assert rc == 0
    expect = {tuple(oracle.lam(wx, i) for wx in w)
              for i in itertools.product(*[range(x) for x in n])}
    got = _enumerate_pairs(P["dims"], 3) if P["dims"] else {(0, 0, 0)}
    assert got == expect


def test_entrywise_kernel_choice(tl):
    n = (64, 64, 64)
    F, L = (1, 2, 3), (3, 2, 1)
    # mixed layouts whose extents and strides allow 16-byte vectors take the
    # vector tile kernel (FP32 and FP64)
    for dtype, tile in (("f32", "ew_tile"), ("f64", "ew_tile")):
        for pa, pb, pc, kern in [(F, F, F, "ew_flat"), (F, L, F, tile), (L, F, F, tile),
                                 (L, L, L, "ew_flat")]:
            rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, n, pa, dtype=dtype),
                          _desc(tl, n, pc, dtype=dtype, addr=FAKE * 4096),
                          B=_desc(tl, n, pb, dtype=dtype, addr=FAKE * 8192), eop=tl.TL_ADD)
            assert rc == 0 and P["kernel"] == kern, (dtype, pa, pb, pc, P)
    # permuted rows (every operand contiguous along mode 1) take the rows
    # kernel; FP32 tiles with a ragged extent but 16-byte strides (a padded
    # view) take the TMA-staged kernel
    for dtype in ("f32", "f64"):
        rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, n, F, dtype=dtype),
                      _desc(tl, n, F, dtype=dtype, addr=FAKE * 4096),
                      B=_desc(tl, n, (1, 3, 2), dtype=dtype, addr=FAKE * 8192), eop=tl.TL_ADD)
        assert rc == 0 and P["kernel"] == "ew_rows", P
    nr = (61, 64, 64)
    rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, nr, w=(1, 64, 4096)),
                  _desc(tl, nr, w=(1, 64, 4096), addr=FAKE * 4096),
                  B=_desc(tl, nr, w=(64, 1, 4096), addr=FAKE * 8192), eop=tl.TL_ADD)
    assert rc == 0 and P["kernel"] == "ew_tma" and P["tdim"] == 1, P
    rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, nr, w=(1, 64, 4096), dtype="f64"),
                  _desc(tl, nr, w=(1, 64, 4096), dtype="f64", addr=FAKE * 4096),
                  B=_desc(tl, nr, w=(64, 1, 4096), dtype="f64", addr=FAKE * 8192), eop=tl.TL_ADD)
    assert rc == 0 and P["kernel"] == "ew_tile" and P["vec"] == 1, P
    # FP32 but beyond the tensor-map rank (6 dims that do not collapse), or
    # with strides that are not multiples of 16 bytes: the older kernels
    n6 = (8, 3, 2, 3, 2, 4)
    rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, n6, (1, 2, 3, 4, 5, 6)),
                  _desc(tl, n6, (1, 6, 5, 4, 3, 2), addr=FAKE * 4096), eop=tl.TL_COPY)
    assert rc == 0 and P["kernel"] == "ew_rows", P
    rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, (63, 61, 3), (1, 2, 3)),
                  _desc(tl, (63, 61, 3), (2, 1, 3), addr=FAKE * 4096), eop=tl.TL_COPY)
    assert rc == 0 and P["kernel"] == "ew_tile", P
    # tiles of small extents would be mostly empty: every element is mapped
    rc, P = _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, (5, 7, 3), (1, 2, 3)),
                  _desc(tl, (5, 7, 3), (2, 1, 3), addr=FAKE * 4096), eop=tl.TL_COPY)
    assert rc == 0 and P["kernel"] == "ew_generic", P


def test_validation_errors(tl):
    n = (4, 5, 6)
    A = _desc(tl, n)
    C = _desc(tl, (4, 6), addr=FAKE * 4096)
    assert _plan(tl, tl.TL_OP_TTV, A, C, q=2)[0] == 0
    assert _plan(tl, tl.TL_OP_TTV, A, C, q=0)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_TTV, A, C, q=4)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_TTV, A, C, q=1)[0] == tl.TL_EINVAL       # wrong output shape
    assert _plan(tl, tl.TL_OP_TTV, _desc(tl, n, (1, 1, 2)), C, q=2)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_TTV, _desc(tl, (4,)), _desc(tl, (1,), addr=FAKE * 4096), q=1)[0] \
        == tl.TL_EINVAL                                                 # p < 2
    assert _plan(tl, tl.TL_OP_TTV, A, _desc(tl, (4, 6), dtype="f64", addr=FAKE * 4096),
                 q=2)[0] == tl.TL_EINVAL                                # dtype mismatch
    assert _plan(tl, tl.TL_OP_TTV, A, _desc(tl, (4, 6), addr=FAKE), q=2)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_TTV, A, _desc(tl, (4, 6), w=(1, 2), addr=FAKE * 4096),
                 q=2)[0] == tl.TL_EINVAL                                # self-overlapping C
    assert _plan(tl, tl.TL_OP_TTV, _desc(tl, n, w=(1, 0, 3)), C, q=2)[0] == tl.TL_EINVAL
    # empty tensors (an extent of 0) and orders beyond the maximum are rejected
    assert _plan(tl, tl.TL_OP_TTV, _desc(tl, (4, 0, 6)), C, q=2)[0] == tl.TL_EINVAL
    n17 = (1,) * 17
    assert _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, n17), _desc(tl, n17, addr=FAKE * 4096),
                 eop=tl.TL_COPY)[0] == tl.TL_EINVAL
    n16 = (1,) * 16
    assert _plan(tl, tl.TL_OP_ENTRYWISE, _desc(tl, n16), _desc(tl, n16, addr=FAKE * 4096),
                 eop=tl.TL_COPY)[0] == 0
    # ttm
    Cm = _desc(tl, (4, 3, 6), addr=FAKE * 4096)
    assert _plan(tl, tl.TL_OP_TTM, A, Cm, q=2, J=3)[0] == 0
    assert _plan(tl, tl.TL_OP_TTM, A, Cm, q=2, J=4)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_TTM, A, Cm, q=2, J=3, prec=tl.TL_P_F64)[0] == tl.TL_EUNSUPPORTED
    Ad = _desc(tl, n, dtype="f64")
    Cd = _desc(tl, (4, 3, 6), dtype="f64", addr=FAKE * 4096)
    assert _plan(tl, tl.TL_OP_TTM, Ad, Cd, q=2, J=3, prec=tl.TL_P_BF16X3)[0] == tl.TL_EUNSUPPORTED
    assert _plan(tl, tl.TL_OP_TTM, Ad, Cd, q=2, J=3, prec=9)[0] == tl.TL_EINVAL
    # entrywise: B required for binary ops, forbidden for unary ones
    Ce = _desc(tl, n, addr=FAKE * 4096)
    assert _plan(tl, tl.TL_OP_ENTRYWISE, A, Ce, eop=tl.TL_ADD)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_ENTRYWISE, A, Ce, B=_desc(tl, n), eop=tl.TL_COPY)[0] == tl.TL_EINVAL
    assert _plan(tl, tl.TL_OP_ENTRYWISE, A, Ce, eop=tl.TL_COPY)[0] == 0
    # in place with identical descriptors is allowed, with another layout it is not
    assert _plan(tl, tl.TL_OP_ENTRYWISE, A, _desc(tl, n), B=_desc(tl, n, addr=FAKE * 8192),
                 eop=tl.TL_ADD)[0] == 0
    assert _plan(tl, tl.TL_OP_ENTRYWISE, A, _desc(tl, n, (3, 2, 1)),
                 B=_desc(tl, n, addr=FAKE * 8192), eop=tl.TL_ADD)[0] == tl.TL_EINVAL


# ------------------------------------------------------------------ views ---

def test_view_descriptor_matches_the_oracle(tl):
    # tl_view is pointer arithmetic only: the base address is never touched
    g = synth.rng(77)
    base = 1 << 40
    for trial in range(40):
        p = int(g.integers(1, 6))
        n = tuple(int(g.integers(1, 12)) for _ in range(p))
        pi = synth.random_layout(p, g)
        w = oracle.strides(n, pi)
        f = [int(g.integers(0, x)) for x in n]
        l = [int(g.integers(a, x)) for a, x in zip(f, n)]
        t = [int(g.integers(1, 4)) for _ in range(p)]
        A = tl.Desc(base, n, pi, dtype="f64")
        rc, V = tl.tl_view(A, f, t, l)
        assert rc == tl.TL_OK
        nv, wv, gamma = oracle.view(n, w, f, t, l)
        assert V.n == nv and V.w == wv
        assert V.s.data == base + 8 * gamma
        # a view of the view composes (w'' = w' t, Eq. 19)
        f2 = [0] * p
        t2 = [2] * p
        l2 = [x - 1 for x in nv]
        rc, V2 = tl.tl_view(V, f2, t2, l2)
        assert rc == tl.TL_OK
        nv2, wv2, g2 = oracle.view(nv, wv, f2, t2, l2)
        assert V2.n == nv2 and V2.w == wv2 and V2.s.data == V.s.data + 8 * g2


def test_view_paper_example(tl):
    # Sec. 3.3: A of shape (4, 2, 3) first-order; f = (1, 0, 2), t = (2, 1, 1),
    # l = (3, 1, 2) gives n' = (2, 2, 1) and A'(0,0,0) = A(1,0,2)
    A = tl.Desc(4096, (4, 2, 3), dtype="f32")
    rc, V = tl.tl_view(A, (1, 0, 2), (2, 1, 1), (3, 1, 2))
    assert rc == tl.TL_OK and V.n == (2, 2, 1)
    w = oracle.strides((4, 2, 3))
    assert V.s.data == 4096 + 4 * oracle.lam(w, (1, 0, 2))
    # A'(1,1,0) = A(3,1,2)
    assert (V.s.data - 4096) // 4 + oracle.lam(V.w, (1, 1, 0)) == oracle.lam(w, (3, 1, 2))


def test_view_rejects_bad_ranges(tl):
    A = tl.Desc(4096, (4, 2, 3), dtype="f32")
    assert tl.tl_view(A, (0, 0, 0), (0, 1, 1), (3, 1, 2))[0] == tl.TL_EINVAL   # t < 1
    assert tl.tl_view(A, (2, 0, 0), (1, 1, 1), (1, 1, 2))[0] == tl.TL_EINVAL   # f > l
    assert tl.tl_view(A, (0, 0, 0), (1, 1, 1), (4, 1, 2))[0] == tl.TL_EINVAL   # l >= n


# ------------------------------------------ tensor-core ttm launch configuration

def _tc_config(tl, n, q, J, prec=5, pi=None, c_addr=FAKE * 8192, c_pi=None):
    nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
    rc, P = _plan(tl, tl.TL_OP_TTM, _desc(tl, n, pi, addr=FAKE * 4096),
                  _desc(tl, nout, c_pi if c_pi else pi, addr=c_addr), q=q, J=J, prec=prec)
    assert rc == 0 and P["kernel"] == "ttm_tc", P
    return P["tc"]


def test_tc_ring_depth_follows_the_write_share(tl):
    # C as large as A (J = n_q): 4 stages of A in flight per SM, every mode
    for q in (1, 2, 3, 4):
        cfg = _tc_config(tl, (128,) * 4, q, 128)
        assert cfg["a_stages"] == 4 and cfg["b_resident"] == 1, (q, cfg)
    # J = n_q / 4: 4 + 4 * (128 - 32) / 128 = 7 stages
    assert _tc_config(tl, (128,) * 4, 2, 32)["a_stages"] == 7
    # COL tiles of 96 valid rows hold fewer bytes: 4 * 128 / 96 -> 6 stages
    assert _tc_config(tl, (96,) * 4, 2, 96)["a_stages"] == 6
    # 64-row COL tiles: 8
    assert _tc_config(tl, (64,) * 5, 2, 64)["a_stages"] == 8


def test_tc_configuration_fits_the_sm(tl):
    for n, q, J, prec in [((128,) * 4, 1, 128, 5), ((512, 512, 512), 1, 512, 5),
                          ((512, 512, 512), 3, 512, 3), ((512, 512, 512), 1, 64, 4),
                          ((64, 33, 17), 1, 300, 5), ((20, 152, 36), 1, 16, 3)]:
        cfg = _tc_config(tl, n, q, J, prec)
        assert cfg["smem"] <= 227 * 1024, (n, q, J, cfg)
        assert cfg["a_stages"] >= 2 and cfg["op_stages"] >= 2, cfg
        assert cfg["threads"] * 96 <= 65536      # 96 registers per thread fit the SM
    # a converted B above 64 KB streams per k stage instead of staying resident
    assert _tc_config(tl, (512, 512, 512), 1, 512)["b_resident"] == 0
    assert _tc_config(tl, (128,) * 4, 1, 128, prec=3)["b_resident"] == 1   # TF32: 64 KB


def test_tc_store_path_choice(tl):
    n = (128,) * 4
    # 16-byte aligned C with 16-byte strides: TMA stores, both orientations
    assert _tc_config(tl, n, 1, 128)["store"] == "tma"
    assert _tc_config(tl, n, 3, 128)["store"] == "tma"
    # C not 16-byte aligned: the warps store
    assert _tc_config(tl, n, 1, 128, c_addr=FAKE * 8192 + 4)["store"] == "warps"
    assert _tc_config(tl, n, 3, 128, c_addr=FAKE * 8192 + 4)["store"] == "warps"
    # ROW with C rows 37 elements apart: no tensor map
    assert _tc_config(tl, (64, 33, 17), 1, 37)["store"] == "warps"
    assert _tc_config(tl, (64, 33, 17), 1, 40)["store"] == "tma"

"""GPU parity of the batched persistent launch: many ttv / ttm / entrywise
operations of uneven order, extents and layout in one launch, every output
checked against the FP64 oracle, for every per-unit code variant, with CUDA
graph replay and with the autotuner."""
import json
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, TOL, put, rel_err, to_dev

pytestmark = pytest.mark.gpu

# the autotuner's cache for this test module lives in a temporary file
_TUNE = os.path.join(tempfile.mkdtemp(prefix="tlgb_tune_"), "tune.txt")
os.environ.setdefault("TL_TUNE_CACHE", _TUNE)


class OpSet:
    """Random operations (batch recipe, scaled down) with device buffers and
    FP64 oracle references."""

    def __init__(self, tl, dev, count, seed, dtype="f32", max_elems=1 << 13, with_ew=True):
        self.tl, self.dev, self.dtype = tl, dev, dtype
        self.keep, self.ops, self.items = [], [], []
        units = synth.batch_units(count, seed, max_elems=max_elems, pmin=2, pmax=5, emin=2,
                                  emax=24)
        g = synth.rng(seed + 1)
        for i, u in enumerate(units):
            n, pi, q = u.n, u.pi, u.q
            X = synth.normal(n, seed + 100 + i, dtype=np.float64)
            A = put(X, pi, dev, dtype)
            kind = u.op
            if with_ew and i % 5 == 4:
                kind = "entrywise"
            if kind == "ttv":
                nout = tuple(x for r, x in enumerate(n) if r != q - 1)
                pic = synth.random_layout(len(nout), g)
                b = synth.normal((n[q - 1],), seed + 200 + i, dtype=np.float64)
                bt = to_dev(b, dev, dtype)
                C = torch.full((int(np.prod(nout)),), float("nan"), dtype=A.dtype, device=dev)
                DA, DC = tl.Desc(A, n, pi), tl.Desc(C, nout, pic)
                op = tl.make_op(tl.TL_OP_TTV, DA, DC, q=q, vec=bt)
                ref = oracle.ttv(synth.to_memory(np.asarray(X, NP[dtype]), pi), n,
                                 oracle.strides(n, pi), q, b.astype(NP[dtype]),
                                 wC=oracle.strides(nout, pic))
                self.keep += [A, bt, C, DA, DC]
                self.items.append((C, ref))
            elif kind == "ttm":
                J = max(u.J, 1)
                nout = tuple(J if r == q - 1 else x for r, x in enumerate(n))
                pic = synth.random_layout(len(n), g)
                Bm = synth.normal((J, n[q - 1]), seed + 300 + i, dtype=np.float64)
                Bt = to_dev(Bm.reshape(-1), dev, dtype)
                C = torch.full((int(np.prod(nout)),), float("nan"), dtype=A.dtype, device=dev)
                DA, DC = tl.Desc(A, n, pi), tl.Desc(C, nout, pic)
                op = tl.make_op(tl.TL_OP_TTM, DA, DC, q=q, vec=Bt, J=J, ldb_row=n[q - 1],
                                ldb_col=1, precision=tl.TL_P_DEFAULT)
                ref = oracle.ttm(synth.to_memory(np.asarray(X, NP[dtype]), pi), n,
                                 oracle.strides(n, pi), q, Bm.reshape(-1).astype(NP[dtype]), J,
                                 n[q - 1], 1, wC=oracle.strides(nout, pic))
                self.keep += [A, Bt, C, DA, DC]
                self.items.append((C, ref))
            else:
                Y = synth.normal(n, seed + 400 + i, dtype=np.float64)
                pib, pic = synth.random_layout(len(n), g), synth.random_layout(len(n), g)
                Bd = put(Y, pib, dev, dtype)
                C = torch.full((int(np.prod(n)),), float("nan"), dtype=A.dtype, device=dev)
                DA, DB, DC = tl.Desc(A, n, pi), tl.Desc(Bd, n, pib), tl.Desc(C, n, pic)
                op = tl.make_op(tl.TL_OP_ENTRYWISE, DA, DC, B=DB, entry_op=tl.TL_SUB)
                ref = oracle.entrywise(oracle.OP_SUB, n,
                                       synth.to_memory(np.asarray(X, NP[dtype]), pi),
                                       oracle.strides(n, pi),
                                       synth.to_memory(np.asarray(Y, NP[dtype]), pib),
                                       oracle.strides(n, pib), wC=oracle.strides(n, pic))
                self.keep += [A, Bd, C, DA, DB, DC]
                self.items.append((C, ref))
            self.ops.append(op)

    def reset_outputs(self):
        for C, _ in self.items:
            C.fill_(float("nan"))

    def check(self):
        torch.cuda.synchronize()
        worst = 0.0
        for C, ref in self.items:
            got = C.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got)), "an output element was not written"
            worst = max(worst, rel_err(got, ref))
        assert worst <= TOL[self.dtype], worst
        return worst


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_matches_oracle_default_plan(tl, cuda_dev, dtype):
    s = OpSet(tl, cuda_dev, 240, 7000, dtype)
    rc, b = tl.tl_batch_create(s.ops, 0)
    tl.check(rc, "tl_batch_create")
    try:
        rc, js = tl.tl_batch_describe(b)
        info = json.loads(js)
        assert info["ops"] + info["direct"] == len(s.ops)
        tl.check(tl.tl_batch_run(b))
        s.check()
    finally:
        tl.tl_batch_destroy(b)


@pytest.mark.parametrize("variant,unit", [("TTV_COL", 7), ("TTV_COL", 1000), ("TTV_ROW4", 5),
                                          ("TTV_ROW8", 300), ("TTV_ROW32", 64), ("TTV_VEC", 6),
                                          ("TTV_VEC", 4096)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_every_ttv_variant(tl, cuda_dev, variant, unit, dtype):
    # contractions of 2-24: every remainder of the 8-long (FP32) and 4-long
    # (FP64) load chunks of the ttv units
    s = OpSet(tl, cuda_dev, 120, 7100, dtype)
    rc, b = tl.tl_batch_create(s.ops, 0)
    tl.check(rc)
    try:
        tl.check(tl.tl_batch_set_variant(b, tl.TL_OP_TTV, getattr(tl, "TL_BV_" + variant), unit))
        tl.check(tl.tl_batch_run(b))
        s.check()
    finally:
        tl.tl_batch_destroy(b)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("variant", ["TTM_32", "TTM_64", "TTM_SMALL"])
def test_batch_every_ttm_variant(tl, cuda_dev, dtype, variant):
    s = OpSet(tl, cuda_dev, 120, 7200, dtype)
    rc, b = tl.tl_batch_create(s.ops, 0)
    tl.check(rc)
    try:
        tl.check(tl.tl_batch_set_variant(b, tl.TL_OP_TTM, getattr(tl, "TL_BV_" + variant), 1))
        tl.check(tl.tl_batch_set_variant(b, tl.TL_OP_ENTRYWISE, tl.TL_BV_EW, 333))
        tl.check(tl.tl_batch_run(b))
        s.check()
    finally:
        tl.tl_batch_destroy(b)


def test_batch_graph_replay_sees_new_data(tl, cuda_dev):
    s = OpSet(tl, cuda_dev, 100, 7300, "f32", with_ew=False)
    rc, b = tl.tl_batch_create(s.ops, tl.TL_BATCH_GRAPH)
    tl.check(rc)
    try:
        for _ in range(2):
            s.reset_outputs()
            tl.check(tl.tl_batch_run(b))
            s.check()
        # scale every A by 2 in place: the replayed graph must see it
        for t in s.keep[0::5]:
            t.mul_(2.0)
        s.reset_outputs()
        tl.check(tl.tl_batch_run(b))
        torch.cuda.synchronize()
        for C, ref in s.items:
            assert rel_err(C.cpu().numpy(), 2.0 * ref) <= TOL["f32"]
    finally:
        tl.tl_batch_destroy(b)


def test_batch_autotuner_choice_is_correct_and_cached(tl, cuda_dev):
    s = OpSet(tl, cuda_dev, 150, 7400, "f32")
    rc, b = tl.tl_batch_create(s.ops, tl.TL_BATCH_TUNE | tl.TL_BATCH_GRAPH)
    tl.check(rc)
    try:
        s.reset_outputs()
        tl.check(tl.tl_batch_run(b))
        s.check()
    finally:
        tl.tl_batch_destroy(b)
    path = os.environ["TL_TUNE_CACHE"]
    assert os.path.exists(path)
    with open(path) as fh:
        lines = [ln.split() for ln in fh if ln.strip()]
    assert lines and all(len(ln) == 3 for ln in lines)
    # a second batch of the same classes is planned from the cache
    rc, b2 = tl.tl_batch_create(s.ops, tl.TL_BATCH_TUNE)
    tl.check(rc)
    try:
        s.reset_outputs()
        tl.check(tl.tl_batch_run(b2))
        s.check()
    finally:
        tl.tl_batch_destroy(b2)


def test_batch_takes_large_tensor_core_ops_directly(tl, cuda_dev):
    n = (64, 33, 17)
    X = synth.normal(n, 7500, dtype=np.float64)
    A = put(X, (1, 2, 3), cuda_dev, "f32")
    Bm = synth.normal((48, 64), 7501, dtype=np.float64)
    Bt = to_dev(Bm.reshape(-1), cuda_dev, "f32")
    C = torch.empty(48 * 33 * 17, dtype=torch.float32, device=cuda_dev)
    DA, DC = tl.Desc(A, n), tl.Desc(C, (48, 33, 17))
    op = tl.make_op(tl.TL_OP_TTM, DA, DC, q=1, vec=Bt, J=48, ldb_row=64, ldb_col=1,
                    precision=tl.TL_P_BF16X3)
    rc, b = tl.tl_batch_create([op], 0)
    tl.check(rc)
    try:
        info = json.loads(tl.tl_batch_describe(b)[1])
        assert info["direct"] == 1 and info["ops"] == 0
        tl.check(tl.tl_batch_run(b))
        torch.cuda.synchronize()
        ref = oracle.ttm(synth.to_memory(X.astype(np.float32), (1, 2, 3)), n, oracle.strides(n), 1,
                         Bm.reshape(-1).astype(np.float32), 48, 64, 1)
        assert rel_err(C.cpu().numpy(), ref) <= 1e-5
    finally:
        tl.tl_batch_destroy(b)


def test_bounded_wait_reports_timeout_and_context_survives(tl, cuda_dev):
    assert tl.tl_device_status() == tl.TL_OK
    tl.check(tl.tl_selftest_wait_timeout(1000.0))
    assert tl.tl_device_status() == tl.TL_ETIMEOUT
    assert tl.tl_device_status() == tl.TL_OK          # cleared by the first report
    s = OpSet(tl, cuda_dev, 20, 7600, "f32")
    rc, b = tl.tl_batch_create(s.ops, 0)
    tl.check(rc)
    try:
        tl.check(tl.tl_batch_run(b))
        s.check()
    finally:
        tl.tl_batch_destroy(b)


_POISON_CHILD = r"""
import json, os, sys
sys.path[:0] = [{tests!r}, {root!r}]
import torch
import paper_1711_10912_gb300 as tl
tl.load_library()
from test_batch_gpu import OpSet
dev = torch.device("cuda", 0)
s = OpSet(tl, dev, 160, 7700, "f32")
rc, b = tl.tl_batch_create(s.ops, tl.TL_BATCH_TUNE)
tl.check(rc)
rc, desc = tl.tl_batch_describe(b)
tl.check(rc)
print(desc, flush=True)
# the host check comes first: a unit that does not fit its operation is never run
if json.loads(desc)["unfit"] != 0:
    sys.exit(3)
tl.check(tl.tl_batch_run(b))
worst = s.check()
tl.tl_batch_destroy(b)
print(json.dumps({{"worst": worst}}))
"""


def test_batch_poisoned_tune_cache_is_ignored(tl, cuda_dev, tmp_path):
    # a cache whose entries name units that do not fit (vectorised ttv and
    # shared-memory ttm everywhere, ragged unit sizes) must not change results:
    # each choice is checked against the operation it is applied to
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, TL_TUNE_CACHE=str(cache))
    code = _POISON_CHILD.format(tests=here, root=os.path.dirname(here))
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
    assert first.returncode == 0, first.stderr[-2000:]
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.strip()]
    assert lines
    poisoned = []
    for key, variant, unit in lines:
        v = tl.TL_BV_TTV_VEC if "|k0|" in key else (tl.TL_BV_TTM_SMALL if "|k1|" in key else variant)
        poisoned.append(f"{key} {v} 6")
    cache.write_text("\n".join(poisoned) + "\n")
    second = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                            timeout=600)
    out = second.stdout.strip().splitlines()
    # the host-side description was printed before the run and shows every
    # poisoned choice replaced
    assert out and json.loads(out[0])["unfit"] == 0, second.stdout[-2000:]
    assert second.returncode == 0, second.stderr[-2000:]
    assert json.loads(out[-1])["worst"] <= TOL["f32"]


def test_batch_keeps_row_unit_ttm_persistent_up_to_256mb(tl, cuda_dev):
    # a 48 MB ttm whose matrix fits the row unit (n_q = 4, J = 8) runs as
    # units of the persistent launch; a 20 MB ttv still runs on its own kernel
    # (16 MB rule); both match the oracle
    n = (4, 1024, 1024)
    X = synth.normal(n, 7600, dtype=np.float64)
    A = put(X, (1, 2, 3), cuda_dev, "f32")
    Bm = synth.normal((8, 4), 7601, dtype=np.float64)
    Bt = to_dev(Bm.reshape(-1), cuda_dev, "f32")
    b = synth.normal((4,), 7602, dtype=np.float64)
    bt = to_dev(b, cuda_dev, "f32")
    Cm = torch.empty(8 * 1024 * 1024, dtype=torch.float32, device=cuda_dev)
    Cv = torch.empty(1024 * 1024, dtype=torch.float32, device=cuda_dev)
    DA, DCm, DCv = tl.Desc(A, n), tl.Desc(Cm, (8, 1024, 1024)), tl.Desc(Cv, (1024, 1024))
    opm = tl.make_op(tl.TL_OP_TTM, DA, DCm, q=1, vec=Bt, J=8, ldb_row=4, ldb_col=1)
    opv = tl.make_op(tl.TL_OP_TTV, DA, DCv, q=1, vec=bt)
    rc, bh = tl.tl_batch_create([opm, opv], 0)
    tl.check(rc)
    try:
        info = json.loads(tl.tl_batch_describe(bh)[1])
        assert info["direct"] == 1 and info["ops"] == 1, info
        tl.check(tl.tl_batch_run(bh))
        torch.cuda.synchronize()
        mem = synth.to_memory(X.astype(np.float32), (1, 2, 3))
        refm = oracle.ttm(mem, n, oracle.strides(n), 1, Bm.reshape(-1).astype(np.float32), 8, 4, 1)
        refv = oracle.ttv(mem, n, oracle.strides(n), 1, b.astype(np.float32))
        assert rel_err(Cm.cpu().numpy(), refm) <= 1e-5
        assert rel_err(Cv.cpu().numpy(), refv) <= 1e-5
    finally:
        tl.tl_batch_destroy(bh)

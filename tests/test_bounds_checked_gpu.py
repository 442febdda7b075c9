"""The bounds-checked debug build (libtlgb_checked.so, TL_CHECK_BOUNDS): every
offset the kernels' index mappers produce is compared with its operand's
extent, and an offset outside is recorded, replaced by one inside and
reported by tl_device_status() as TL_EBOUNDS.

Run in child processes that load the checked library (TL_LIBRARY):
 - small parity cases through every mapper-based kernel path (ttv row,
   staged, column and split-K; ttm tiles, rows, FP32 register tiles and
   split-K; entrywise flat, tiled, rows and generic; norm; a batch of mixed
   operations) must match the FP64 oracle with no violation recorded;
 - with TL_DEBUG_SHRINK_LIMITS set, every limit handed to the kernels is
   halved, so accesses that are in fact inside the operands are reported: the
   check is shown to fire, and since a reported access is redirected to the
   operand's first element, nothing outside the buffers is touched."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

_CHILD = r'''
import sys
sys.path[:0] = [{tests!r}, {root!r}]
import numpy as np
import torch
import paper_1711_10912_gb300 as tl
tl.load_library()
assert tl.tl_bounds_checked() == 1
import oracle
import synth
from gpu_util import TOL, rel_err, ttm_case, ttv_case, put
from test_batch_gpu import OpSet
dev = torch.device("cuda", 0)
g = synth.rng(9900)
worst = 0.0
cases = [((64, 300), 2, (1, 2)), ((300, 64), 1, (1, 2)), ((512, 40), 1, (1, 2)),
         ((5, 9, 130), 2, (3, 1, 2)), ((3, 70000), 2, (1, 2)), ((17, 33, 8, 5), 3, (4, 2, 1, 3))]
for n, q, pi in cases:
    for dtype in ("f32", "f64"):
        X = synth.normal(n, 9901, dtype=np.float64)
        b = synth.normal((n[q - 1],), 9902, dtype=np.float64)
        got, ref = ttv_case(tl, dev, X, q, b, pi, synth.random_layout(len(n) - 1, g), dtype)
        worst = max(worst, rel_err(got, ref) / TOL[dtype])
        for J in (7, 40, 300):
            Bm = synth.normal((J, n[q - 1]), 9903 + J, dtype=np.float64)
            got, ref = ttm_case(tl, dev, X, q, Bm, pi, synth.random_layout(len(n), g), dtype)
            worst = max(worst, rel_err(got, ref) / TOL[dtype])
for n in ((64, 96), (33, 17, 9), (8, 9, 10, 11)):
    p = len(n)
    X = synth.normal(n, 9904, dtype=np.float64)
    Y = synth.normal(n, 9905, dtype=np.float64)
    for pa, pb, pc in ((synth.first_order(p),) * 3, (synth.first_order(p), synth.last_order(p),
                        synth.first_order(p)), (synth.random_layout(p, g), synth.random_layout(p, g),
                                                synth.random_layout(p, g))):
        for dtype in ("f32", "f64"):
            A, B = put(X, pa, dev, dtype), put(Y, pb, dev, dtype)
            C = torch.empty(int(np.prod(n)), dtype=A.dtype, device=dev)
            tl.check(tl.tl_entrywise(tl.TL_SUB, tl.Desc(A, n, pa), tl.Desc(B, n, pb), 0.0,
                                     tl.Desc(C, n, pc)))
            torch.cuda.synchronize()
            got = synth.from_memory(C.cpu().numpy(), n, pc)
            assert np.array_equal(got, (X.astype(A.cpu().numpy().dtype) -
                                        Y.astype(A.cpu().numpy().dtype)))
            r = torch.zeros(3, dtype=torch.float64, device=dev)
            tl.check(tl.tl_norm(tl.Desc(A, n, pa), r))
            torch.cuda.synchronize()
            want = np.linalg.norm(X.astype(A.cpu().numpy().dtype).astype(np.float64))
            assert abs(float(r[0]) - want) <= 1e-12 * want
s = OpSet(tl, dev, 120, 9906, "f32")
rc, bt = tl.tl_batch_create(s.ops, 0)
tl.check(rc)
tl.check(tl.tl_batch_run(bt))
s.check()
tl.tl_batch_destroy(bt)
status = tl.tl_device_status()
print("worst/tol", worst, "status", status)
assert worst <= 1.0, worst
assert status == tl.TL_OK, status
print("CHECKED_OK")
'''

_PLANTED = r'''
import sys
sys.path[:0] = [{tests!r}, {root!r}]
import numpy as np
import torch
import paper_1711_10912_gb300 as tl
tl.load_library()
assert tl.tl_bounds_checked() == 1
from test_batch_gpu import OpSet
dev = torch.device("cuda", 0)
A = torch.randn(64 * 300, device=dev)
b = torch.randn(300, device=dev)
C = torch.empty(64, device=dev)
tl.check(tl.tl_ttv(tl.Desc(A, (64, 300)), b, 1, 2, tl.Desc(C, (64,))))
first = tl.tl_device_status()
assert tl.tl_device_status() == tl.TL_OK        # the word was cleared
s = OpSet(tl, dev, 40, 9907, "f32")
rc, bt = tl.tl_batch_create(s.ops, 0)
tl.check(rc)
tl.check(tl.tl_batch_run(bt))
second = tl.tl_device_status()
tl.tl_batch_destroy(bt)
print("statuses", first, second)
assert first == tl.TL_EBOUNDS and second == tl.TL_EBOUNDS
print("PLANTED_OK")
'''


def _run(code, extra_env):
    from paper_1711_10912_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, TL_LIBRARY=lib, **extra_env)
    return subprocess.run([sys.executable, "-c", code.format(tests=HERE, root=ROOT)], env=env,
                          capture_output=True, text=True, timeout=900)


def test_checked_build_parity_without_violations(tl, cuda_dev):
    r = _run(_CHILD, {})
    assert r.returncode == 0 and "CHECKED_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]


def test_checked_build_reports_planted_violations(tl, cuda_dev):
    r = _run(_PLANTED, {"TL_DEBUG_SHRINK_LIMITS": "1"})
    assert r.returncode == 0 and "PLANTED_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]

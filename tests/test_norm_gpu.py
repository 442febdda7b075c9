"""GPU parity of tl_norm (Table 3, norm) and tl_rel_error against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import put, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("seed", range(6))
def test_norm_random_layouts(tl, cuda_dev, dtype, seed):
    g = synth.rng(4000 + seed)
    p = int(g.integers(1, 6))
    n = tuple(int(x) for x in g.integers(1, 30, size=p))
    X = synth.normal(n, 4100 + seed, dtype=np.float64)
    pi = synth.random_layout(p, g)
    A = put(X, pi, cuda_dev, dtype)
    res = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_norm(tl.Desc(A, n, pi), res))
    torch.cuda.synchronize()
    ref = oracle.norm(A.cpu().numpy(), n, oracle.strides(n, pi))
    assert abs(res[0].item() - ref) <= 1e-13 * ref


def test_norm_large_deterministic(tl, cuda_dev):
    n = (301, 257, 19)
    X = synth.normal(n, 4200, dtype=np.float64)
    A = put(X, (2, 1, 3), cuda_dev, "f64")
    res = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    vals = []
    for _ in range(3):
        tl.check(tl.tl_norm(tl.Desc(A, n, (2, 1, 3)), res))
        torch.cuda.synchronize()
        vals.append(res[0].item())
    assert vals[0] == vals[1] == vals[2]
    ref = oracle.norm(A.cpu().numpy(), n, oracle.strides(n, (2, 1, 3)))
    assert abs(vals[0] - ref) <= 1e-13 * ref


def test_rel_error_mixed_dtypes_and_layouts(tl, cuda_dev):
    n = (40, 33, 7)
    R = synth.normal(n, 4300, dtype=np.float64)
    Xl = (R * (1 + 1e-3)).astype(np.float32)
    Xd = put(Xl, (3, 2, 1), cuda_dev, "f32")
    Rd = put(R, (1, 2, 3), cuda_dev, "f64")
    res = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_rel_error(tl.Desc(Xd, n, (3, 2, 1)), tl.Desc(Rd, n), res))
    torch.cuda.synchronize()
    ref = oracle.rel_error(Xd.cpu().numpy(), oracle.strides(n, (3, 2, 1)), Rd.cpu().numpy(),
                           oracle.strides(n), n)
    assert abs(res[0].item() - ref) <= 1e-12 * ref
    assert abs(res[0].item() - 1e-3) < 1e-6

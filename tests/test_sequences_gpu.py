"""GPU parity of the chained operations of Sec. 5.2 Table 3 (times_vectors,
times_matrices) and of the higher-order power method listed there, through the
C ABI, against the FP64 oracle's ttvs / ttms / hopm on the same seeded
inputs."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NP, TOL, TORCH, get, put, rel_err, to_dev

pytestmark = pytest.mark.gpu

TTVS_CASES = [
    ((37, 20, 9), (2, 3), (1, 2, 3), (1,)),
    ((37, 20, 9), (1, 3), (3, 1, 2), (1,)),
    ((12, 7, 33, 5), (1, 2, 4), (4, 2, 1, 3), (1,)),
    ((12, 7, 33, 5), (4, 2), (2, 4, 3, 1), (2, 1)),
    ((6, 5, 4, 3, 7), (5, 1, 3), (5, 4, 3, 2, 1), (1, 2)),
    ((300, 64, 3), (2,), (1, 2, 3), (2, 1)),
    ((65, 129, 2), (2, 3), (2, 3, 1), (1,)),
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,modes,pi,pic", TTVS_CASES)
def test_ttvs_matches_oracle(tl, cuda_dev, dtype, n, modes, pi, pic):
    X = synth.uniform(n, 600 + len(n) + sum(modes))
    vecs = [synth.uniform((n[m - 1],), 700 + m) for m in modes]
    A = put(X, pi, cuda_dev, dtype)
    vd = [to_dev(v, cuda_dev, dtype) for v in vecs]
    rest = tuple(x for r, x in enumerate(n) if r + 1 not in modes)
    C = torch.full((int(np.prod(rest)),), float("nan"), dtype=TORCH[dtype], device=cuda_dev)
    tl.check(tl.tl_ttvs(tl.Desc(A, n, pi), vd, modes, tl.Desc(C, rest, pic)), "tl_ttvs")
    torch.cuda.synchronize()
    Xd = np.asarray(X, NP[dtype])
    ref, rn = oracle.ttvs(synth.to_memory(Xd, pi), n, oracle.strides(n, pi), modes,
                          [np.asarray(v, NP[dtype]) for v in vecs])
    assert rn == rest
    assert rel_err(get(C, rest, pic), synth.from_memory(ref, rest, tuple(range(1, len(rest) + 1)))) \
        <= TOL[dtype]


def test_ttvs_on_a_subtensor_view(tl, cuda_dev):
    # A is the view [2:30, 1:19, 3:9, 0:4] of a 32x20x10x4 first-order tensor (Eq. 18)
    big = (32, 20, 10, 4)
    X = synth.uniform(big, 640)
    mem = synth.to_memory(X, (1, 2, 3, 4))
    wb = oracle.strides(big)
    lo = (2, 1, 3, 0)
    n = (28, 18, 6, 4)
    off = int(sum(l * w for l, w in zip(lo, wb)))
    Abig = to_dev(mem, cuda_dev, "f64")
    modes = (1, 3)
    vecs = [synth.uniform((n[m - 1],), 650 + m) for m in modes]
    vd = [to_dev(v, cuda_dev, "f64") for v in vecs]
    rest = (18, 4)
    C = torch.empty(18 * 4, dtype=torch.float64, device=cuda_dev)
    DA = tl.Desc(Abig.data_ptr() + 8 * off, n, w=wb, dtype=torch.float64)
    tl.check(tl.tl_ttvs(DA, vd, modes, tl.Desc(C, rest)))
    torch.cuda.synchronize()
    ref, _ = oracle.ttvs(mem, n, wb, modes, vecs, offA=off)
    assert rel_err(C.cpu().numpy(), ref) <= TOL["f64"]


def test_ttvs_rejects_bad_calls(tl, cuda_dev):
    n = (4, 5, 6)
    A = torch.zeros(120, dtype=torch.float32, device=cuda_dev)
    v = [torch.zeros(x, dtype=torch.float32, device=cuda_dev) for x in n]
    C1 = torch.zeros(6, dtype=torch.float32, device=cuda_dev)
    DA = tl.Desc(A, n)
    assert tl.tl_ttvs(DA, v, (1, 2, 3), tl.Desc(C1, (1,))) == tl.TL_EINVAL   # no mode left
    assert tl.tl_ttvs(DA, v[:2], (1, 1), tl.Desc(C1, (6,))) == tl.TL_EINVAL  # repeated mode
    assert tl.tl_ttvs(DA, v[:2], (1, 4), tl.Desc(C1, (6,))) == tl.TL_EINVAL  # out of range
    assert tl.tl_ttvs(DA, v[:2], (1, 2), tl.Desc(C1, (5,))) == tl.TL_EINVAL  # wrong C extent
    assert tl.tl_ttvs(DA, [], (), tl.Desc(C1, (6,))) == tl.TL_EINVAL          # nothing to do


TTMS_CASES = [
    ((24, 17, 9), (1, 2, 3), (7, 5, 3), (1, 2, 3), "f64", 0),
    ((24, 17, 9), (3, 1), (4, 30), (3, 1, 2), "f64", 0),
    ((10, 6, 8, 5), (2, 4), (9, 2), (2, 4, 1, 3), "f32", 0),
    ((128, 64, 40), (1, 2, 3), (32, 16, 8), (1, 2, 3), "f32", 5),
    ((96, 80, 24), (2, 1), (64, 48), (1, 2, 3), "f32", 2),
]


@pytest.mark.parametrize("n,modes,J,pi,dtype,prec", TTMS_CASES)
def test_ttms_matches_oracle(tl, cuda_dev, n, modes, J, pi, dtype, prec):
    X = synth.uniform(n, 800 + len(modes))
    mats = [synth.uniform((j, n[m - 1]), 810 + m) for m, j in zip(modes, J)]
    A = put(X, pi, cuda_dev, dtype)
    md = [to_dev(M.reshape(-1), cuda_dev, dtype) for M in mats]
    nout = list(n)
    for m, j in zip(modes, J):
        nout[m - 1] = j
    nout = tuple(nout)
    C = torch.full((int(np.prod(nout)),), float("nan"), dtype=TORCH[dtype], device=cuda_dev)
    tl.check(tl.tl_ttms(tl.Desc(A, n, pi), md, J, modes, tl.Desc(C, nout, pi), prec), "tl_ttms")
    torch.cuda.synchronize()
    ref, rn = oracle.ttms(synth.to_memory(np.asarray(X, NP[dtype]), pi), n,
                          oracle.strides(n, pi), modes, [np.asarray(M, NP[dtype]) for M in mats])
    assert rn == nout
    assert rel_err(get(C, nout, pi), synth.from_memory(ref, nout, tuple(range(1, len(n) + 1)))) \
        <= TOL[dtype]


def test_ttms_tucker_projection_of_the_precision_workload(tl, cuda_dev):
    # the all-modes 512^3 -> 64^3 projection in one call
    n, mem, B, Bt, U = synth.precision_case()
    A = torch.from_numpy(mem).to(cuda_dev)
    Ud = [torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).to(cuda_dev) for u in U]
    C = torch.empty(64 ** 3, dtype=torch.float32, device=cuda_dev)
    tl.check(tl.tl_ttms(tl.Desc(A, n), Ud, (64, 64, 64), (1, 2, 3), tl.Desc(C, (64, 64, 64)),
                        tl.TL_P_BF16X3))
    torch.cuda.synchronize()
    # sampled outputs against the closed form C = A x1 U1 x2 U2 x3 U3 in FP64,
    # evaluated as three plain matrix products (first-order storage: X[k, j, i])
    g = synth.rng(820)
    idx = np.stack([g.integers(0, 64, size=256) for _ in range(3)], axis=1)
    X = mem.reshape(512 * 512, 512).astype(np.float64)
    T = (X @ U[0].astype(np.float64).T).reshape(512, 512, 64)          # [k, j, a]
    T = np.matmul(U[1].astype(np.float64), T)                          # [k, b, a]
    T = (U[2].astype(np.float64) @ T.reshape(512, 64 * 64)).reshape(64, 64, 64)  # [c, b, a]
    got = C.cpu().numpy().reshape(64, 64, 64)
    sel = (idx[:, 2], idx[:, 1], idx[:, 0])
    assert rel_err(got[sel], T[sel]) <= 1e-5
    # and the oracle's own ttms agrees on a reduced copy (first 64 of every mode)
    small = np.ascontiguousarray(mem.reshape(512, 512, 512)[:64, :64, :64]).reshape(-1)
    As = torch.from_numpy(small).to(cuda_dev)
    Us = [np.ascontiguousarray(u[:, :64]) for u in U]
    Usd = [torch.from_numpy(u.reshape(-1)).to(cuda_dev) for u in Us]
    Cs = torch.empty(64 ** 3, dtype=torch.float32, device=cuda_dev)
    tl.check(tl.tl_ttms(tl.Desc(As, (64, 64, 64)), Usd, (64, 64, 64), (1, 2, 3),
                        tl.Desc(Cs, (64, 64, 64)), tl.TL_P_BF16X3))
    torch.cuda.synchronize()
    refs, _ = oracle.ttms(small, (64, 64, 64), oracle.strides((64, 64, 64)), (1, 2, 3), Us)
    assert rel_err(Cs.cpu().numpy(), refs) <= 1e-5


def test_ttms_rejects_bad_calls(tl, cuda_dev):
    n = (4, 5, 6)
    A = torch.zeros(120, dtype=torch.float64, device=cuda_dev)
    M = torch.zeros(64, dtype=torch.float64, device=cuda_dev)
    C = torch.zeros(120, dtype=torch.float64, device=cuda_dev)
    DA = tl.Desc(A, n)
    assert tl.tl_ttms(DA, [M, M], (4, 5), (1, 1), tl.Desc(C, n)) == tl.TL_EINVAL
    assert tl.tl_ttms(DA, [M], (3,), (2,), tl.Desc(C, n)) == tl.TL_EINVAL     # C keeps n_2
    assert tl.tl_ttms(DA, [M], (0,), (2,), tl.Desc(C, (4, 0, 6))) == tl.TL_EINVAL


def _rank1_plus_noise(n, seed, eps):
    vs = [synth.uniform((x,), seed + r) for r, x in enumerate(n)]
    vs = [v / np.linalg.norm(v) for v in vs]
    sigma = 3.0
    X = sigma * vs[0]
    for v in vs[1:]:
        X = np.multiply.outer(X, v)
    return X + eps * synth.uniform(n, seed + 50), vs, sigma


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,pi", [((20, 30, 12), (1, 2, 3)), ((9, 14, 6, 11), (3, 1, 4, 2)),
                                  ((5, 6, 4, 3, 7), (5, 3, 1, 2, 4)), ((200, 150), (2, 1))])
def test_hopm_matches_oracle(tl, cuda_dev, dtype, n, pi):
    X, _, _ = _rank1_plus_noise(n, 900 + len(n), 0.05)
    u0 = [synth.uniform((x,), 950 + r) for r, x in enumerate(n)]
    A = put(X, pi, cuda_dev, dtype)
    ud = [to_dev(u, cuda_dev, dtype) for u in u0]
    lam = torch.zeros(len(n), dtype=torch.float64, device=cuda_dev)
    K = 4
    tl.check(tl.tl_hopm(tl.Desc(A, n, pi), ud, lam, K), "tl_hopm")
    torch.cuda.synchronize()
    ru, rl = oracle.hopm(synth.to_memory(np.asarray(X, NP[dtype]), pi), n, oracle.strides(n, pi),
                         [np.asarray(u, NP[dtype]) for u in u0], K)
    tol = TOL[dtype] * 10
    assert rel_err(lam.cpu().numpy(), rl) <= tol
    for got, ref in zip(ud, ru):
        assert rel_err(got.cpu().numpy(), ref) <= tol


def test_hopm_rank_one_tensor_gives_sigma_in_one_sweep(tl, cuda_dev):
    # for an exact rank-1 tensor sigma * v1 o v2 o v3 the first sweep already
    # turns every u_r into +-v_r, so the second returns lambda_r = sigma for all r
    n = (40, 25, 33)
    X, vs, sigma = _rank1_plus_noise(n, 970, 0.0)
    A = put(X, (1, 2, 3), cuda_dev, "f64")
    ud = [to_dev(synth.uniform((x,), 980 + r), cuda_dev, "f64") for r, x in enumerate(n)]
    lam = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    tl.check(tl.tl_hopm(tl.Desc(A, n), ud, lam, 2))
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    assert np.all(np.abs(lam - sigma) <= 1e-12 * sigma)
    for r in range(3):
        u = ud[r].cpu().numpy()
        assert min(np.linalg.norm(u - vs[r]), np.linalg.norm(u + vs[r])) <= 1e-12


def test_sequences_leave_the_device_status_clean(tl, cuda_dev):
    assert tl.tl_device_status() == tl.TL_OK

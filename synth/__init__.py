"""Seeded synthetic inputs for the ttv / ttm / entrywise workloads.

This module only draws random numbers and lays logical numpy arrays out in
memory; it holds none of the method's arithmetic.  Both the oracle-side tests
and the CUDA-side tests / benchmark take their inputs from here, so the two
sides see identical data.

Memory layout of a logical array X with extents n under the 1-based layout
tuple pi (pi[0] is the fastest-varying mode) is produced with numpy's own
transpose + C-order ravel: the axes are listed slowest first, i.e.
(pi[p-1]-1, ..., pi[0]-1).  This is numpy's notion of storage order, not a
restatement of the paper's stride formula, so tests can use it to pin the
oracle's layout function independently.

Workload recipes (sizes, distributions) follow the five configurations the
project measures: a small order-3 FP64 case, an order-4 128^4 FP32 bandwidth
study, a 512^3 precision study, a 4096-tensor batch and a Poisson serving
stream.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1711


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def first_order(p: int) -> tuple:
    return tuple(range(1, p + 1))


def last_order(p: int) -> tuple:
    return tuple(range(p, 0, -1))


def random_layout(p: int, g: np.random.Generator) -> tuple:
    return tuple(int(x) + 1 for x in g.permutation(p))


def all_layouts(p: int):
    return [tuple(x) for x in itertools.permutations(range(1, p + 1))]


def _axes_slowest_first(pi) -> list:
    return [int(r) - 1 for r in reversed(tuple(pi))]


def to_memory(X: np.ndarray, pi) -> np.ndarray:
    """Storage-order 1-D buffer of logical array X in layout pi."""
    if X.ndim == 0:
        return X.reshape(1).copy()
    return np.ascontiguousarray(np.transpose(X, _axes_slowest_first(pi))).reshape(-1)


def from_memory(mem: np.ndarray, n, pi) -> np.ndarray:
    """Inverse of to_memory: the logical array held by a dense buffer."""
    n = tuple(int(x) for x in n)
    axes = _axes_slowest_first(pi)
    Y = np.asarray(mem).reshape([n[a] for a in axes])
    return np.transpose(Y, np.argsort(axes))


def uniform(shape, seed: int, lo=-1.0, hi=1.0, dtype=np.float64) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=shape).astype(dtype)


def normal(shape, seed: int, scale=1.0, dtype=np.float32) -> np.ndarray:
    g = rng(seed)
    if np.dtype(dtype) == np.float32:
        x = g.standard_normal(size=shape, dtype=np.float32)
        if scale != 1.0:
            x *= np.float32(scale)
        return x
    return (g.standard_normal(size=shape) * scale).astype(dtype)


def integers(shape, seed: int, lo=-8, hi=8, dtype=np.float64) -> np.ndarray:
    """Small integers in [lo, hi]: products and sums stay exact in FP32/FP64."""
    return rng(seed).integers(lo, hi + 1, size=shape).astype(dtype)


# ------------------------------------------------------------ workloads ---

@dataclass
class SmallCase:
    """Order-3 FP64 64x64x64, first-order layout, U[-1,1]; ttv along mode 2
    with a length-64 vector, ttm along mode 1 with a 32x64 matrix, entrywise
    add with a last-order copy of the same tensor."""
    n: tuple
    X: np.ndarray          # logical array, float64
    b: np.ndarray          # length n[1]
    B: np.ndarray          # 32 x n[0], row-major
    q_ttv: int = 2
    q_ttm: int = 1


def small_case(seed: int = BASE_SEED + 1) -> SmallCase:
    n = (64, 64, 64)
    X = uniform(n, seed)
    b = uniform((n[1],), seed + 100)
    B = uniform((32, n[0]), seed + 200)
    return SmallCase(n=n, X=X, b=b, B=B)


@dataclass
class ScaleCase:
    """Order-4 FP32 128^4 (1 GiB) with N(0,1) entries; per-mode vectors of
    length 128 and 128x128 matrices N(0,1)/sqrt(128)."""
    n: tuple
    mem_first: np.ndarray  # storage of the logical tensor in first-order layout
    vectors: list          # b_q, q = 1..4
    matrices: list         # B_q, q = 1..4 (128 x 128, row-major)


def scale_case(seed: int = BASE_SEED + 2, edge: int = 128, order: int = 4) -> ScaleCase:
    n = (edge,) * order
    N = edge ** order
    mem = normal((N,), seed, dtype=np.float32)
    vecs = [normal((edge,), seed + 10 + q, dtype=np.float32) for q in range(order)]
    mats = [normal((edge, edge), seed + 20 + q, scale=1.0 / math.sqrt(edge), dtype=np.float32)
            for q in range(order)]
    return ScaleCase(n=n, mem_first=mem, vectors=vecs, matrices=mats)


def precision_case(seed: int = BASE_SEED + 3, edge: int = 512, rank: int = 64):
    """Order-3 edge^3 FP32 N(0,1) whose mode-3 slices are scaled by
    10^u_k, u_k ~ U(-3,3); a edge x edge N(0,1) matrix, its first `rank`
    rows as the truncated matrix, and three rank x edge Tucker factors
    N(0,1)/sqrt(edge).  Returns (n, logical-first-order memory, B, Bt, U)."""
    n = (edge, edge, edge)
    g = rng(seed)
    mem = g.standard_normal(size=edge ** 3, dtype=np.float32)
    u = g.uniform(-3.0, 3.0, size=edge)
    scale = (10.0 ** u).astype(np.float32)
    # first-order storage: mode 3 is the slowest, so slice k is a contiguous block
    mem.reshape(edge, edge * edge)[:] *= scale[:, None]
    B = normal((edge, edge), seed + 1, dtype=np.float32)
    Bt = np.ascontiguousarray(B[:rank])
    U = [normal((rank, edge), seed + 2 + r, scale=1.0 / math.sqrt(edge), dtype=np.float32)
         for r in range(3)]
    return n, mem, B, Bt, U


@dataclass
class BatchUnit:
    op: str                # "ttv" or "ttm"
    n: tuple
    pi: tuple
    q: int
    J: int = 0             # rows of the matrix for ttm


def batch_units(count: int = 4096, seed: int = BASE_SEED + 4, max_elems: int = 1 << 20,
                pmin: int = 3, pmax: int = 6, emin: int = 4, emax: int = 64):
    """Batch recipe: order p ~ U{3..6}; each extent log-uniform in [4, 64]
    and rounded; the draw is repeated until prod(n) <= 2^20; layout uniform
    over all p! permutations; mode q ~ U{1..p}; 50% ttv / 50% ttm with the
    matrix row count log-uniform in [4, 64]."""
    g = rng(seed)
    units = []
    lo, hi = math.log(emin), math.log(emax)
    for _ in range(count):
        p = int(g.integers(pmin, pmax + 1))
        while True:
            n = tuple(int(round(math.exp(g.uniform(lo, hi)))) for _ in range(p))
            if math.prod(n) <= max_elems:
                break
        pi = random_layout(p, g)
        q = int(g.integers(1, p + 1))
        if g.uniform() < 0.5:
            units.append(BatchUnit("ttv", n, pi, q))
        else:
            J = int(round(math.exp(g.uniform(lo, hi))))
            units.append(BatchUnit("ttm", n, pi, q, J))
    return units


@dataclass
class Request:
    t_arrive: float        # seconds from stream start
    op: str                # "ttv", "ttm" or "entrywise"
    n: tuple
    pi: tuple
    q: int
    dtype: str             # "f32" or "f64"
    J: int = 0
    pi_b: tuple = ()       # layout of the second entrywise operand
    pi_c: tuple = ()       # layout of the output
    seed: int = 0


def _split_extents(g, N: float, p: int, nmin: int = 2) -> tuple:
    """Splits log(N) across p modes by Dirichlet(1) weights; n_r >= nmin."""
    wts = g.dirichlet(np.ones(p))
    n = [max(nmin, int(round(math.exp(math.log(N) * w)))) for w in wts]
    return tuple(n)


def serving_stream(count: int, rate: float, seed: int = BASE_SEED + 5,
                   log10_mean: float = 5.5, log10_sd: float = 1.25,
                   log10_lo: float = 3.0, log10_hi: float = 8.0):
    """Poisson request stream: exponential inter-arrival times at `rate`
    requests/s; op mix 40% ttv / 40% ttm / 20% entrywise; order p ~ U{2..7};
    log10 of the element count ~ N(5.5, 1.25) truncated to [3, 8] and split
    across modes; 80% FP32 / 20% FP64; random layouts and modes."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += g.exponential(1.0 / rate)
        u = g.uniform()
        op = "ttv" if u < 0.4 else ("ttm" if u < 0.8 else "entrywise")
        p = int(g.integers(2, 8))
        while True:
            z = g.normal(log10_mean, log10_sd)
            if log10_lo <= z <= log10_hi:
                break
        n = _split_extents(g, 10.0 ** z, p)
        pi = random_layout(p, g)
        q = int(g.integers(1, p + 1))
        dt = "f64" if g.uniform() < 0.2 else "f32"
        J = int(round(math.exp(g.uniform(math.log(4), math.log(64))))) if op == "ttm" else 0
        pib = random_layout(p, g) if op == "entrywise" else ()
        pic = random_layout(p, g) if op == "entrywise" else ()
        out.append(Request(t, op, n, pi, q, dt, J, pib, pic, seed=int(g.integers(1 << 31))))
    return out


def device_normal(torch, count: int, seed: int, dtype, device):
    """N(0,1) values generated on the device from a seeded torch generator
    (for operands too large to draw on the host quickly)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn(int(count), generator=g, dtype=dtype, device=device)

"""The request-serving runtime: continuous batching of ttv / ttm / entrywise
requests with admission against a memory budget.

Checks that every result served in a mix of concurrent requests is
bit-identical to the same request served alone, and within tolerance of the
FP64 oracle; that the budget is never exceeded while several batches are
launched; that oversized requests are rejected; and that queued requests can
be cancelled."""
import time

import numpy as np
import pytest
import torch

from test_batch_gpu import OpSet
from gpu_util import TOL

pytestmark = pytest.mark.gpu


def serve_all(tl, ctx, ops, gap_s=0.0):
    tickets = []
    for o in ops:
        rc, t = tl.tl_batch_submit(ctx, [o])
        tl.check(rc, "tl_batch_submit")
        tickets.append(t)
        if gap_s:
            time.sleep(gap_s)
    lat = []
    for t in tickets:
        rc, st, ms = tl.tl_wait(ctx, t, 60000.0)
        tl.check(rc, "tl_wait")
        assert st == tl.TL_OK
        lat.append(ms)
    return lat


@pytest.mark.parametrize("flags", [1, 0])
def test_results_same_alone_and_in_the_mix(tl, cuda_dev, flags):
    s = OpSet(tl, cuda_dev, 160, 8000, "f32")
    s64 = OpSet(tl, cuda_dev, 40, 8100, "f64")
    ops = s.ops + s64.ops
    items = s.items + s64.items
    rc, ctx = tl.tl_ctx_create(1 << 30, 3, flags)
    tl.check(rc, "tl_ctx_create")
    try:
        # alone: one request at a time
        alone = []
        for o, (C, _) in zip(ops, items):
            C.fill_(float("nan"))
            serve_all(tl, ctx, [o])
            torch.cuda.synchronize()
            alone.append(C.cpu().numpy().copy())
        # in the mix: everything submitted at once
        for C, _ in items:
            C.fill_(float("nan"))
        serve_all(tl, ctx, ops)
        torch.cuda.synchronize()
        for (C, ref), a in zip(items, alone):
            got = C.cpu().numpy()
            np.testing.assert_array_equal(got, a)
        s.check()
        s64.check()
        rc, max_inflight, batches, completed = tl.tl_ctx_stats(ctx)
        assert completed == 2 * len(ops)
        assert batches < 2 * len(ops)        # the mix was batched
    finally:
        tl.tl_ctx_destroy(ctx)


def test_budget_bounds_inflight_bytes(tl, cuda_dev):
    s = OpSet(tl, cuda_dev, 120, 8200, "f32")
    budget = 3 * 8 * 8192 * 4        # a few of the largest requests at once
    rc, ctx = tl.tl_ctx_create(budget, 4, tl.TL_CTX_PERSISTENT)
    tl.check(rc)
    try:
        serve_all(tl, ctx, s.ops)
        s.check()
        rc, max_inflight, batches, completed = tl.tl_ctx_stats(ctx)
        assert 0 < max_inflight <= budget
        assert batches > 1 and completed == len(s.ops)
    finally:
        tl.tl_ctx_destroy(ctx)


def test_oversized_request_is_rejected(tl, cuda_dev):
    s = OpSet(tl, cuda_dev, 4, 8300, "f32")
    rc, ctx = tl.tl_ctx_create(64, 1, tl.TL_CTX_PERSISTENT)
    tl.check(rc)
    try:
        rc, _ = tl.tl_batch_submit(ctx, [s.ops[0]])
        assert rc == tl.TL_ENOMEM
    finally:
        tl.tl_ctx_destroy(ctx)


def test_queued_request_can_be_cancelled(tl, cuda_dev):
    s = OpSet(tl, cuda_dev, 60, 8400, "f32")
    # a budget of one request at a time keeps the tail of the queue waiting
    big = max(int(np.prod(C.shape)) for C, _ in s.items)
    rc, ctx = tl.tl_ctx_create(1, 1, tl.TL_CTX_PERSISTENT) if False else \
        tl.tl_ctx_create(16 * big * 4 + (1 << 16), 1, tl.TL_CTX_PERSISTENT)
    tl.check(rc)
    try:
        tickets = []
        for o in s.ops:
            rc, t = tl.tl_batch_submit(ctx, [o])
            tl.check(rc)
            tickets.append(t)
        rc = tl.tl_cancel(ctx, tickets[-1])
        assert rc in (tl.TL_OK, tl.TL_PENDING)
        for t in tickets[:-1]:
            rc, st, _ = tl.tl_wait(ctx, t, 60000.0)
            assert rc == tl.TL_OK and st == tl.TL_OK
        rc, st, _ = tl.tl_wait(ctx, tickets[-1], 60000.0)
        assert rc == tl.TL_OK and st in (tl.TL_ECANCELED, tl.TL_OK)
        # a reported ticket is forgotten
        assert tl.tl_poll(ctx, tickets[0])[0] == tl.TL_EINVAL
    finally:
        tl.tl_ctx_destroy(ctx)

"""Failure paths of the plan workspaces, driven on the host (no GPU fault):
dct_debug_fail_alloc makes the n-th allocation attempt of a workspace fail
as out-of-memory.  Every call that meets it must return DCT_ERR_ALLOC with
nothing enqueued, free what it had allocated, and leave the plan usable:
the same call then succeeds and gives the results of a clean plan."""
import numpy as np
import pytest
import torch

from synth import powerlaw_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    yield dctgb
    dctgb.dct_debug_fail_alloc(0)


def srcs_and_quals():
    rng = np.random.default_rng(17)
    srcs = [powerlaw_image(int(rng.integers(8, 90)), int(rng.integers(8, 90)), seed=400 + i, device="cuda")
            for i in range(5)]
    return srcs, [int(q) for q in rng.integers(10, 96, size=5)]


def attempts_of(D, fn):
    before = D.dct_debug_fail_alloc(0)
    fn()
    return D.dct_debug_fail_alloc(0) - before


def test_batch_workspace_allocation_failures(D):
    srcs, quals = srcs_and_quals()
    S = D.DCT_OP_SSE                       # the fused pass that stores nothing but the SSE
    ref = torch.zeros(5, dtype=torch.int64, device="cuda")
    with D.Plan(128, 128, max_batch=8) as plan:
        k = attempts_of(D, lambda: D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals), S, sse=ref))
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
    assert k == 8                        # 4 device buffers, 3 pinned buffers, 1 stream
    for n in range(1, k + 1):
        sse = torch.full((5,), -1, dtype=torch.int64, device="cuda")
        with D.Plan(128, 128, max_batch=8) as plan:
            D.dct_debug_fail_alloc(n)
            with pytest.raises(D.DctError) as ei:
                D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals), S, sse=sse)
            assert ei.value.status == 3, n
            torch.cuda.synchronize()
            assert int(sse.min()) == -1 and int(sse.max()) == -1       # nothing was enqueued
            with pytest.raises(D.DctError) as ei:
                D.dct_batch_launch(plan)                                 # nothing prepared
            assert ei.value.status == 6
            D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals), S, sse=sse)
            D.dct_batch_launch(plan)
            torch.cuda.synchronize()
            assert torch.equal(sse, ref), n


def test_autotune_event_failure_keeps_the_plan(D):
    srcs, quals = srcs_and_quals()
    S = D.DCT_OP_SSE
    sse = torch.zeros(5, dtype=torch.int64, device="cuda")
    with D.Plan(128, 128, max_batch=8) as plan:
        D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals), S, sse=sse)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        ref = sse.clone()
        for n in (1, 2):                                                 # the two timing events
            D.dct_debug_fail_alloc(n)
            with pytest.raises(D.DctError) as ei:
                D.dct_autotune(plan)
            assert ei.value.status == 3
        D.dct_debug_fail_alloc(3)                                        # the flush buffer: timed warm instead
        D.dct_autotune(plan)
        D.dct_debug_fail_alloc(0)
        sse.fill_(-1)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        assert torch.equal(sse, ref)


def test_rate_control_workspace_allocation_failures(D):
    imgs = [powerlaw_image(40 + 8 * i, 48, seed=500 + i, device="cuda") for i in range(3)]
    targets = [30.0, 34.0, 38.0]
    with D.Plan(96, 96, max_batch=4) as plan:
        k = attempts_of(D, lambda: D.dct_rate_control(plan, imgs, 1, targets))
    with D.Plan(96, 96, max_batch=4) as plan:
        ref = D.dct_rate_control(plan, imgs, 1, targets)
    assert k > 20
    for n in sorted({1, 2, k // 2, k - 1, k}):
        with D.Plan(96, 96, max_batch=4) as plan:
            D.dct_debug_fail_alloc(n)
            with pytest.raises(D.DctError) as ei:
                D.dct_rate_control(plan, imgs, 1, targets)
            assert ei.value.status == 3, n
            got = D.dct_rate_control(plan, imgs, 1, targets)
            assert np.array_equal(got["quality"], ref["quality"]) and np.array_equal(got["sse"], ref["sse"]), n

"""The allocation-free batch entry point (dct_batch_run_noalloc).

It is for callers that cannot allocate device memory while they run (device
memory reserved up front by another allocator, loops that cannot absorb the
device synchronisation of cudaMalloc / cudaFree, fixed memory budgets).  It
keeps its work list in a fixed array inside the library instead of plan
memory, so these tests check that it gives exactly what the plan-based path
gives, twice in a row (the array is reused), and that it refuses batches
larger than that array.  The file is named to run last: a failure here
leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from synth import powerlaw_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def batch(seed, n):
    rng = np.random.default_rng(seed)
    srcs, quals, chroma = [], [], []
    for i in range(n):
        h, w = int(rng.integers(8, 260)), int(rng.integers(8, 260))
        srcs.append(powerlaw_image(h, w, seed=seed * 1000 + i, beta=float(rng.uniform(1, 3)), device="cuda"))
        quals.append(int(rng.integers(1, 101)))
        chroma.append(bool(rng.integers(0, 2)))
    return srcs, quals, chroma


def outputs(D, srcs, fill):
    coefs = [torch.full((D.coeff_count([s.shape]),), fill, dtype=torch.int16, device="cuda") for s in srcs]
    recs = [torch.full_like(s, fill & 0xFF) for s in srcs]
    sse = torch.full((len(srcs),), -1, dtype=torch.int64, device="cuda")
    return coefs, recs, sse


@pytest.mark.parametrize("ops_name", ["fused", "two_pass", "compress"])
def test_noalloc_matches_plan_path_twice(D, ops_name):
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    ops = {"fused": C | R | S, "two_pass": C | R | S | T, "compress": C}[ops_name]
    srcs, quals, chroma = batch(7, 40)
    # reference: the plan-based batched path
    rc, rr, rs = outputs(D, srcs, 0)
    with D.Plan(512, 512, max_batch=64) as plan:
        items = D.make_batch_items(srcs, quals, coeffs=rc, recons=rr, chroma=chroma)
        D.dct_batch_prepare(plan, items, ops, sse=rs if ops & S else None)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
    for call in range(2):
        nc, nr, ns = outputs(D, srcs, 77 + call)
        items = D.make_batch_items(srcs, quals, coeffs=nc, recons=nr, chroma=chroma)
        D.dct_batch_run_noalloc(items, ops, sse=ns if ops & S else None)
        torch.cuda.synchronize()
        for i in range(len(srcs)):
            assert torch.equal(nc[i], rc[i]), (call, i)
            if ops & R:
                assert torch.equal(nr[i], rr[i]), (call, i)
        if ops & S:
            assert torch.equal(ns, rs), call


def test_noalloc_custom_tables_and_limits(D):
    rng = np.random.default_rng(8)
    srcs, quals, _ = batch(9, 6)
    tabs = [rng.integers(1, 256, size=64) for _ in srcs]
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    rc, rr, rs = outputs(D, srcs, 0)
    with D.Plan(512, 512, max_batch=8) as plan:
        D.dct_batch_prepare(plan, D.make_batch_items(srcs, [0] * 6, coeffs=rc, recons=rr, qtabs=tabs), C | R | S,
                            sse=rs)
        D.dct_batch_launch(plan)
    nc, nr, ns = outputs(D, srcs, 5)
    D.dct_batch_run_noalloc(D.make_batch_items(srcs, [0] * 6, coeffs=nc, recons=nr, qtabs=tabs), C | R | S, sse=ns)
    torch.cuda.synchronize()
    assert torch.equal(ns, rs)
    assert all(torch.equal(a, b) for a, b in zip(nc, rc))
    # 65 items is one more than the fixed work list holds
    t = torch.zeros(8, 8, dtype=torch.uint8, device="cuda")
    c = torch.zeros(64, dtype=torch.int16, device="cuda")
    with pytest.raises(D.DctError) as ei:
        D.dct_batch_run_noalloc(D.make_batch_items([t] * 65, [50] * 65, coeffs=[c] * 65), C)
    assert ei.value.status == 1 and "64" in str(ei.value)

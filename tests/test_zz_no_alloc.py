"""The allocation-free batch entry point (dct_batch_run_noalloc).

It is for callers that cannot allocate device memory while they run: a
process whose device memory another allocator reserved up front, a loop that
cannot absorb the device synchronisation of cudaMalloc / cudaFree, or a
deployment with a fixed memory budget.  It keeps its work list in a fixed
array inside the library instead of plan memory, so these tests check that
it gives exactly what the plan-based path gives, twice in a row (the array
is reused), for every operation mode and for the largest batch the array
holds; that one call matches the CPU oracle directly; that it leaves the
device's free memory unchanged; that it refuses batches larger than its
array; and that it refuses to run on a stream that is being captured (its
descriptors come from the caller's stack).  The file is named to run last:
a failure here leaves every other test already run.
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


def batch(seed, n, lo=8, hi=260):
    rng = np.random.default_rng(seed)
    srcs, quals, chroma = [], [], []
    for i in range(n):
        h, w = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        srcs.append(powerlaw_image(h, w, seed=seed * 1000 + i, beta=float(rng.uniform(1, 3)), device="cuda"))
        quals.append(int(rng.integers(1, 101)))
        chroma.append(bool(rng.integers(0, 2)))
    return srcs, quals, chroma


def outputs(D, srcs, fill):
    coefs = [torch.full((D.coeff_count([s.shape]),), fill, dtype=torch.int16, device="cuda") for s in srcs]
    recs = [torch.full_like(s, fill & 0xFF) for s in srcs]
    sse = torch.full((len(srcs),), -1, dtype=torch.int64, device="cuda")
    return coefs, recs, sse


OPS = ["fused", "two_pass", "compress", "compress_sse", "sse_only", "reconstruct", "reconstruct_sse"]


def ops_of(D, name):
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    return {"fused": C | R | S, "two_pass": C | R | S | T, "compress": C, "compress_sse": C | S, "sse_only": S,
            "reconstruct": R, "reconstruct_sse": R | S}[name]


def run_both(D, ops, srcs, quals, chroma, calls=2):
    """Plan path once, then dct_batch_run_noalloc `calls` times; yields each
    call's outputs next to the plan path's.  The reconstruct-only modes read
    the coefficients the plan path's compress pass wrote."""
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    rc, rr, rs = outputs(D, srcs, 0)
    with D.Plan(512, 512, max_batch=64) as plan:
        if not ops & C and ops & R:
            D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals, coeffs=rc, chroma=chroma), C)
            D.dct_batch_launch(plan)
        D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals, coeffs=rc, recons=rr, chroma=chroma), ops,
                            sse=rs if ops & S else None)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
    for call in range(calls):
        nc, nr, ns = outputs(D, srcs, 77 + call)
        if not ops & C and ops & R:
            nc = [c.clone() for c in rc]               # coefficients in
        items = D.make_batch_items(srcs, quals, coeffs=nc, recons=nr, chroma=chroma)
        D.dct_batch_run_noalloc(items, ops, sse=ns if ops & S else None)
        torch.cuda.synchronize()
        yield call, (rc, rr, rs), (nc, nr, ns)


@pytest.mark.parametrize("ops_name", OPS)
def test_noalloc_matches_plan_path_twice(D, ops_name):
    ops = ops_of(D, ops_name)
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    srcs, quals, chroma = batch(7, 40)
    for call, (rc, rr, rs), (nc, nr, ns) in run_both(D, ops, srcs, quals, chroma):
        for i in range(len(srcs)):
            if ops & C:
                assert torch.equal(nc[i], rc[i]), (call, i)
            if ops & R:
                assert torch.equal(nr[i], rr[i]), (call, i)
        if ops & S:
            assert torch.equal(ns, rs), call
            assert int(ns.min()) >= 0


def test_noalloc_largest_batch(D):
    """64 items, the size of the static work list, in the fused mode."""
    srcs, quals, chroma = batch(21, 64, 8, 130)
    for call, (rc, rr, rs), (nc, nr, ns) in run_both(D, ops_of(D, "fused"), srcs, quals, chroma):
        assert torch.equal(ns, rs), call
        assert all(torch.equal(a, b) for a, b in zip(nc, rc)), call
        assert all(torch.equal(a, b) for a, b in zip(nr, rr)), call


def test_noalloc_matches_the_oracle(D):
    """One call checked directly against the CPU oracle: codes, reconstruction and SSE."""
    from oracle import codec, ijg, psnr
    srcs, quals, chroma = batch(33, 5, 8, 90)
    coefs, recs, sse = outputs(D, srcs, 3)
    D.dct_batch_run_noalloc(D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs, chroma=chroma),
                            ops_of(D, "fused"), sse=sse)
    torch.cuda.synchronize()
    for i, s in enumerate(srcs):
        img = s.cpu().numpy()
        Q = ijg.chroma_table(quals[i]) if chroma[i] else ijg.luma_table(quals[i])
        c = codec.compress_plane(img, Q)
        r = codec.reconstruct_plane(c, Q, *img.shape)
        assert np.array_equal(coefs[i].cpu().numpy(), c.reshape(-1)), i
        assert np.array_equal(recs[i].cpu().numpy(), r), i
        assert int(sse[i]) == psnr.sse(img, r), i


def test_noalloc_leaves_device_memory_unchanged(D):
    """After a first call (which may load the library's kernels), further
    calls change neither the device's free memory nor torch's allocations."""
    srcs, quals, chroma = batch(41, 12, 8, 200)
    coefs, recs, sse = outputs(D, srcs, 0)
    items = D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs, chroma=chroma)
    ops = ops_of(D, "two_pass")
    D.dct_batch_run_noalloc(items, ops, sse=sse)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        D.dct_batch_run_noalloc(items, ops, sse=sse)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_noalloc_refused_while_its_stream_is_captured(D):
    """The call returns DCT_ERR_UNSUPPORTED and enqueues nothing while its
    stream is capturing; the capture itself stays valid."""
    srcs, quals, chroma = batch(51, 3, 8, 40)
    coefs, recs, sse = outputs(D, srcs, 0)
    items = D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs, chroma=chroma)
    side = torch.cuda.Stream()
    x = torch.zeros(16, device="cuda")
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        try:
            D.dct_batch_run_noalloc(items, ops_of(D, "fused"), sse=sse, stream=side)
        except D.DctError as e:
            refused = e
    assert refused is not None and refused.status == 2
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    assert int(sse[0]) == -1                      # nothing of the refused call ran


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

"""GPU parity of the batched persistent, graph-captured path: images of
uneven sizes and qualities in one launch, against the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import codec, ijg, psnr
from synth import batch_workload, powerlaw_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def make_items(n, seed, lo=8, hi=300, ragged=True):
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n):
        h = int(rng.integers(lo, hi + 1))
        w = int(rng.integers(lo, hi + 1))
        if not ragged:
            h, w = max(8, h // 8 * 8), max(8, w // 8 * 8)
        q = int(rng.integers(1, 101))
        chroma = bool(rng.integers(0, 2))
        img = powerlaw_image(h, w, seed=seed * 1000 + i, beta=float(rng.uniform(1, 3))).numpy()
        items.append(dict(img=img, quality=q, chroma=chroma))
    return items


def table(it):
    return ijg.chroma_table(it["quality"]) if it["chroma"] else ijg.luma_table(it["quality"])


def oracle(it):
    Q = table(it)
    c = codec.compress_plane(it["img"], Q)
    r = codec.reconstruct_plane(c, Q, *it["img"].shape)
    return c.reshape(-1), r, psnr.sse(it["img"], r)


def run_batch(D, plan, items, ops, shape=None, launches=1):
    srcs = [torch.from_numpy(it["img"]).cuda() for it in items]
    coefs = [torch.full((D.coeff_count([s.shape]),), 12345, dtype=torch.int16, device="cuda") for s in srcs]
    recs = [torch.zeros_like(s) for s in srcs]
    sse = torch.full((len(items),), -1, dtype=torch.int64, device="cuda")
    arr = D.make_batch_items(srcs, [it["quality"] for it in items], coeffs=coefs, recons=recs,
                             chroma=[it["chroma"] for it in items])
    D.dct_batch_prepare(plan, arr, ops, sse=sse if ops & D.DCT_OP_SSE else None, shape=shape)
    for _ in range(launches):
        D.dct_batch_launch(plan)
    torch.cuda.synchronize()
    return coefs, recs, sse, srcs, arr


@pytest.mark.parametrize("shape", [None, (64, 1, 32, 0), (256, 2, 32, 0), (128, 16, 32, 0),
                                   (64, 1, 32, 2), (256, 4, 32, 2), (128, 16, 32, 2)])
def test_batch_fused_matches_oracle(D, shape):
    items = make_items(24, seed=1)
    with D.Plan(512, 512, max_batch=64) as plan:
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        coefs, recs, sse, _, _ = run_batch(D, plan, items, C | R | S, shape=shape)
        for i, it in enumerate(items):
            c_or, r_or, s_or = oracle(it)
            assert np.array_equal(coefs[i].cpu().numpy(), c_or), i
            assert np.array_equal(recs[i].cpu().numpy(), r_or), i
            assert int(sse[i]) == s_or, i


@pytest.mark.parametrize("lanes", [1, 2])
@pytest.mark.parametrize("mode", ["compress", "sse_only", "compress_sse", "recon_sse", "recon_only", "twopass",
                                  "twopass_nosse"])
def test_batch_op_combinations(D, mode, lanes):
    items = make_items(12, seed=2)
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    ops = {"compress": C, "sse_only": S, "compress_sse": C | S, "recon_sse": C | R | S, "recon_only": C | R,
           "twopass": C | R | S | T, "twopass_nosse": C | R | T}[mode]
    with D.Plan(512, 512, max_batch=16) as plan:
        coefs, recs, sse, _, _ = run_batch(D, plan, items, ops, shape=(128, 2, 32, lanes))
        for i, it in enumerate(items):
            c_or, r_or, s_or = oracle(it)
            if ops & C:
                assert np.array_equal(coefs[i].cpu().numpy(), c_or), i
            else:
                assert int((coefs[i] != 12345).sum()) == 0
            if ops & R:
                assert np.array_equal(recs[i].cpu().numpy(), r_or), i
            else:
                assert int(recs[i].abs().sum()) == 0
            if ops & S:
                assert int(sse[i]) == s_or, i


def test_batch_inverse_only_from_coefficients(D):
    items = make_items(10, seed=3)
    with D.Plan(512, 512, max_batch=16) as plan:
        srcs = [torch.from_numpy(it["img"]).cuda() for it in items]
        coefs = [torch.from_numpy(oracle(it)[0]).cuda() for it in items]
        recs = [torch.zeros_like(s) for s in srcs]
        sse = torch.zeros(len(items), dtype=torch.int64, device="cuda")
        arr = D.make_batch_items(srcs, [it["quality"] for it in items], coeffs=coefs, recons=recs,
                                 chroma=[it["chroma"] for it in items])
        D.dct_batch_prepare(plan, arr, D.DCT_OP_RECONSTRUCT | D.DCT_OP_SSE, sse=sse)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        for i, it in enumerate(items):
            _, r_or, s_or = oracle(it)
            assert np.array_equal(recs[i].cpu().numpy(), r_or)
            assert int(sse[i]) == s_or


def test_batch_graph_replay_is_deterministic(D):
    items = make_items(16, seed=4)
    with D.Plan(512, 512, max_batch=16) as plan:
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        coefs, recs, sse, _, _ = run_batch(D, plan, items, C | R | S, launches=1)
        first = (sse.clone(), [c.clone() for c in coefs])
        for _ in range(5):
            D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        assert torch.equal(sse, first[0])
        for a, b in zip(coefs, first[1]):
            assert torch.equal(a, b)


def test_batch_custom_tables_and_single_item(D):
    rng = np.random.default_rng(5)
    img = powerlaw_image(70, 90, seed=5).numpy()
    qt = rng.integers(1, 256, size=64)
    with D.Plan(128, 128, max_batch=1) as plan:
        src = torch.from_numpy(img).cuda()
        coef = torch.empty(D.coeff_count([src.shape]), dtype=torch.int16, device="cuda")
        rec = torch.empty_like(src)
        sse = torch.zeros(1, dtype=torch.int64, device="cuda")
        arr = D.make_batch_items([src], [0], coeffs=[coef], recons=[rec], qtabs=[qt])
        D.dct_batch_prepare(plan, arr, D.DCT_OP_COMPRESS | D.DCT_OP_RECONSTRUCT | D.DCT_OP_SSE, sse=sse)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        Q = qt.reshape(8, 8)
        c_or = codec.compress_plane(img, Q)
        r_or = codec.reconstruct_plane(c_or, Q, 70, 90)
        assert np.array_equal(coef.cpu().numpy(), c_or.reshape(-1))
        assert np.array_equal(rec.cpu().numpy(), r_or)
        assert int(sse[0]) == psnr.sse(img, r_or)


def test_batch_autotune_keeps_results(D):
    items = make_items(20, seed=6, lo=64, hi=400)
    with D.Plan(512, 512, max_batch=32) as plan:
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        coefs, recs, sse, _, arr = run_batch(D, plan, items, C | R | S)
        ref = sse.clone()
        shape, ms = D.dct_autotune(plan)
        assert shape[0] in (64, 128, 256) and shape[1] >= 1 and ms > 0
        sse.fill_(-1)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        assert torch.equal(sse, ref)


def test_batch_workload_shapes_sampled(D):
    """The 512-image batched workload (sizes 64..2048, qualities 10..95):
    every item's SSE against its reconstruction, and sampled items against
    the oracle."""
    spec = batch_workload(512)
    srcs, quals = [], []
    for it in spec:
        srcs.append(powerlaw_image(it["height"], it["width"], seed=it["seed"], beta=it["beta"], device="cuda"))
        quals.append(it["quality"])
    with D.Plan(2048, 2048, max_batch=512) as plan:
        coefs = [torch.empty(D.coeff_count([s.shape]), dtype=torch.int16, device="cuda") for s in srcs]
        recs = [torch.empty_like(s) for s in srcs]
        sse = torch.zeros(512, dtype=torch.int64, device="cuda")
        arr = D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs)
        D.dct_batch_prepare(plan, arr, D.DCT_OP_COMPRESS | D.DCT_OP_RECONSTRUCT | D.DCT_OP_SSE, sse=sse)
        D.dct_autotune(plan)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        for i in range(512):
            d = recs[i].to(torch.int64) - srcs[i].to(torch.int64)
            assert int(sse[i]) == int((d * d).sum())
        for i in (0, 7, 100, 333, 511):
            if srcs[i].numel() > 600_000:
                continue
            it = dict(img=srcs[i].cpu().numpy(), quality=quals[i], chroma=False)
            c_or, r_or, s_or = oracle(it)
            assert np.array_equal(coefs[i].cpu().numpy(), c_or)
            assert np.array_equal(recs[i].cpu().numpy(), r_or)
            assert int(sse[i]) == s_or


def test_batch_invalid_arguments(D):
    t = torch.zeros(16, 16, dtype=torch.uint8, device="cuda")
    c = torch.zeros(4 * 64, dtype=torch.int16, device="cuda")
    with D.Plan(32, 32, max_batch=2) as plan:
        with pytest.raises(D.DctError):   # no prepared batch
            D.dct_batch_launch(plan)
        arr = D.make_batch_items([t, t, t], [50, 50, 50], coeffs=[c, c, c])
        with pytest.raises(D.DctError):   # more than max_batch
            D.dct_batch_prepare(plan, arr, D.DCT_OP_COMPRESS)
        arr = D.make_batch_items([t], [50], coeffs=[c])
        with pytest.raises(D.DctError):   # SSE without sse_out
            D.dct_batch_prepare(plan, arr, D.DCT_OP_SSE)
        with pytest.raises(D.DctError):   # two-pass without reconstruct
            D.dct_batch_prepare(plan, arr, D.DCT_OP_COMPRESS | D.DCT_OP_TWO_PASS)
        with pytest.raises(D.DctError):   # bad shape
            D.dct_batch_prepare(plan, arr, D.DCT_OP_COMPRESS, shape=(100, 1, 32, 0))
    with D.Plan(32, 32, max_batch=0) as plan:
        with pytest.raises(D.DctError):
            D.dct_batch_prepare(plan, D.make_batch_items([t], [50], coeffs=[c]), D.DCT_OP_COMPRESS)


@pytest.mark.parametrize("lanes", [1, 2])
def test_batch_maximum_plane_sampled(D, lanes):
    """The largest plane a plan accepts below 2^31 samples, 32767 x 65535
    (ragged in both directions), through the fused batch in the benchmark's
    launch shapes (one and two lanes per block): the last block row and column and 1024 random interior
    blocks against the oracle, the SSE against the reconstruction."""
    h, w = 32767, 65535
    quality = 50
    gen = torch.Generator(device="cuda")
    gen.manual_seed(65535)
    src = torch.randint(0, 256, (h, w), dtype=torch.uint8, device="cuda", generator=gen)
    nby, nbx = (h + 7) // 8, (w + 7) // 8
    with D.Plan(w, h, max_batch=1) as plan:
        coef = torch.empty(D.coeff_count([src.shape]), dtype=torch.int16, device="cuda")
        rec = torch.empty_like(src)
        sse = torch.zeros(1, dtype=torch.int64, device="cuda")
        arr = D.make_batch_items([src], [quality], coeffs=[coef], recons=[rec])
        D.dct_batch_prepare(plan, arr, D.DCT_OP_COMPRESS | D.DCT_OP_RECONSTRUCT | D.DCT_OP_SSE, sse=sse,
                            shape=(256, 16, 32, lanes))
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
    Q = ijg.luma_table(quality)
    cblk = coef.view(nby, nbx, 8, 8)
    # last block row and last block column: oracle on the edge strips
    for strip, rstrip, idx in ((src[8 * (nby - 1):, :], rec[8 * (nby - 1):, :], (slice(nby - 1, nby), slice(None))),
                               (src[:, 8 * (nbx - 1):], rec[:, 8 * (nbx - 1):], (slice(None), slice(nbx - 1, nbx)))):
        img = strip.cpu().numpy()
        c_or = codec.compress_plane(img, Q)
        assert np.array_equal(cblk[idx].cpu().numpy(), c_or)
        assert np.array_equal(rstrip.cpu().numpy(), codec.reconstruct_plane(c_or, Q, *img.shape))
    # random interior blocks
    rng = np.random.default_rng(3)
    by = torch.from_numpy(rng.integers(0, nby - 1, 1024)).cuda()
    bx = torch.from_numpy(rng.integers(0, nbx - 1, 1024)).cuda()
    r8 = torch.arange(8, device="cuda")
    rows = (8 * by[:, None] + r8)[:, :, None]
    cols = (8 * bx[:, None] + r8)[:, None, :]
    blocks = src[rows, cols].cpu().numpy()
    c_or = codec.compress_blocks(blocks, Q)
    assert np.array_equal(cblk[by, bx].cpu().numpy(), c_or)
    assert np.array_equal(rec[rows, cols].cpu().numpy(), codec.reconstruct_blocks(c_or, Q))
    # SSE of the whole plane, in row chunks
    tot = 0
    for r0 in range(0, h, 4096):
        d = rec[r0:r0 + 4096].to(torch.int32) - src[r0:r0 + 4096].to(torch.int32)
        tot += int((d * d).sum(dtype=torch.int64))
    assert int(sse[0]) == tot


def test_batch_sse_restarts_between_batches(D):
    """Every replay starts the SSE words from zero: replays, a re-prepare
    with fewer items, other launch shapes and an autotune on the same plan
    all give the oracle's SSE."""
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    items_a = make_items(10, seed=21)
    items_b = make_items(4, seed=22)
    with D.Plan(512, 512, max_batch=16) as plan:
        _, _, sse, _, _ = run_batch(D, plan, items_a, C | R | S, launches=3)
        assert [int(v) for v in sse.cpu()] == [oracle(it)[2] for it in items_a]
        for shape in (None, (64, 4, 32, 1), (256, 2, 32, 2)):
            _, _, sse, _, _ = run_batch(D, plan, items_b, S, shape=shape, launches=2)
            assert [int(v) for v in sse.cpu()] == [oracle(it)[2] for it in items_b], shape
        D.dct_autotune(plan)
        sse.fill_(-1)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
        assert [int(v) for v in sse.cpu()] == [oracle(it)[2] for it in items_b]


def test_batch_claimed_chunks_match_one_lane_ranges(D):
    """A small grid over many tiles (at least 16 per warp) makes the two-lane
    kernel claim four tiles at a time; its coefficients, reconstructions and
    SSE equal the one-lane kernel's fixed-range results bit for bit, and
    sampled blocks equal the oracle."""
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    srcs = [powerlaw_image(1600, 1600 - 8 * i, seed=40 + i, device="cuda") for i in range(4)]
    quals = [30, 50, 75, 95]
    out = {}
    with D.Plan(1600, 1600, max_batch=4) as plan:
        for lanes, shape in ((2, (64, 1, 32, 2)), (1, (256, 2, 32, 1))):
            coefs = [torch.empty(D.coeff_count([s.shape]), dtype=torch.int16, device="cuda") for s in srcs]
            recs = [torch.empty_like(s) for s in srcs]
            sse = torch.zeros(4, dtype=torch.int64, device="cuda")
            D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs), C | R | S,
                                sse=sse, shape=shape)
            for _ in range(2):
                D.dct_batch_launch(plan)
            torch.cuda.synchronize()
            out[lanes] = (coefs, recs, sse.clone())
    ntiles = sum((((s.shape[0] + 7) // 8) * ((s.shape[1] + 7) // 8) + 31) // 32 for s in srcs)
    assert ntiles >= 16 * torch.cuda.get_device_properties(0).multi_processor_count * 2   # warps of the small grid
    for a, b in zip(out[2][0] + out[2][1], out[1][0] + out[1][1]):
        assert torch.equal(a, b)
    assert torch.equal(out[2][2], out[1][2])
    it = dict(img=srcs[3][:64, :64].cpu().numpy(), quality=quals[3], chroma=False)
    c_or, r_or, _ = oracle(it)
    nbx = (srcs[3].shape[1] + 7) // 8
    cb = out[2][0][3].view(-1, nbx, 8, 8)[:8, :8].cpu().numpy().reshape(-1)
    assert np.array_equal(cb, c_or)
    assert np.array_equal(out[2][1][3][:64, :64].cpu().numpy(), r_or)


def test_full_size_workload_in_the_benchmark_configuration(D):
    """The benchmark's step exactly: the 8192 x 8192 grey plane and the
    3840 x 2160 4:2:0 frame (quality 75, luma and chroma tables) in one
    fused batch, launch shape from dct_autotune, replayed from the graph:
    sampled blocks (2048 random ones plus the last block row and column of
    each plane) against the oracle and every plane's SSE against its
    reconstruction."""
    import bench
    planes, chroma = bench.make_planes(torch.device("cuda", 0))
    shapes = [tuple(p.shape) for p in planes]
    coefs = [torch.empty(D.coeff_count([s]), dtype=torch.int16, device="cuda") for s in shapes]
    recs = [torch.empty_like(p) for p in planes]
    sse = torch.zeros(len(planes), dtype=torch.int64, device="cuda")
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    with D.Plan(8192, 8192, max_batch=len(planes)) as plan:
        D.dct_batch_prepare(plan, D.make_batch_items(planes, [bench.QUALITY] * 4, coeffs=coefs, recons=recs,
                                                     chroma=chroma), C | R | S, sse=sse)
        shape, _ = D.dct_autotune(plan)
        for _ in range(2):
            D.dct_batch_launch(plan)
        torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    for p, c, r, is_chroma, e in zip(planes, coefs, recs, chroma, sse.cpu().tolist()):
        h, w = p.shape
        nby, nbx = (h + 7) // 8, (w + 7) // 8
        Q = ijg.chroma_table(bench.QUALITY) if is_chroma else ijg.luma_table(bench.QUALITY)
        bys = np.concatenate([rng.integers(0, nby, 2048), np.full(nbx, nby - 1), np.arange(nby)])
        bxs = np.concatenate([rng.integers(0, nbx, 2048), np.arange(nbx), np.full(nby, nbx - 1)])
        sel = np.unique(bys * nbx + bxs)
        blocks = codec.plane_to_blocks(p.cpu().numpy()).reshape(-1, 8, 8)[sel]
        c_or = codec.compress_blocks(blocks, Q)
        got = c.view(-1, 8, 8)[torch.from_numpy(sel).cuda()].cpu().numpy()
        assert np.array_equal(got, c_or)
        r_or = codec.reconstruct_blocks(c_or, Q)
        rec = codec.plane_to_blocks(r.cpu().numpy()).reshape(-1, 8, 8)[sel]
        by_s, bx_s = sel // nbx, sel % nbx
        for k in range(sel.size):
            nr, nc = min(8, h - 8 * by_s[k]), min(8, w - 8 * bx_s[k])
            assert np.array_equal(rec[k, :nr, :nc], r_or[k, :nr, :nc])
        d = r.to(torch.int64) - p.to(torch.int64)
        assert int(e) == int((d * d).sum())

"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer outputs (int16 coefficients, uint8 reconstructions, uint64 SSE and
statistics words) must match bit for bit; PSNR must match to 1e-9 relative
(it is the same function of the same integer SSE)."""
import math

import numpy as np
import pytest
import torch

from oracle import codec, features, ijg, psnr
from synth import powerlaw_image, ragged_sizes, sinusoid_image, yuv420_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def rand_img(h, w, seed):
    rng = np.random.default_rng(seed)
    kind = seed % 3
    if kind == 0:
        return rng.integers(0, 256, size=(h, w), dtype=np.uint8)
    if kind == 1:
        return powerlaw_image(h, w, seed).numpy()
    return sinusoid_image(h, w, seed).numpy()


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_roundtrip(img, Q):
    c = codec.compress_plane(img, Q)
    r = codec.reconstruct_plane(c, Q, *img.shape)
    return c.reshape(-1), r, psnr.sse(img, r)


@pytest.mark.parametrize("quality", [1, 10, 50, 75, 95, 100])
def test_compress_reconstruct_ragged(D, quality):
    Q = ijg.luma_table(quality)
    with D.Plan(1024, 1024) as plan:
        for k, (h, w) in enumerate(ragged_sizes()):
            img = rand_img(h, w, 100 * quality + k)
            c_or, r_or, s_or = oracle_roundtrip(img, Q)
            t = gpu(img)
            coef = D.dct_compress(plan, [t], quality)
            out = torch.empty_like(t)
            sse = D.dct_reconstruct(plan, coef, [out], quality, ref_planes=[t])
            torch.cuda.synchronize()
            assert np.array_equal(coef.cpu().numpy(), c_or), (h, w)
            assert np.array_equal(out.cpu().numpy(), r_or), (h, w)
            assert int(sse.cpu()[0]) == s_or, (h, w)


@pytest.mark.parametrize("quality", [5, 50, 90])
def test_fused_matches_oracle_and_two_call(D, quality):
    Q = ijg.luma_table(quality)
    with D.Plan(2048, 2048) as plan:
        for k, (h, w) in enumerate([(8, 8), (37, 29), (264, 8), (200, 200), (257, 511)]):
            img = rand_img(h, w, 7 * quality + k)
            c_or, r_or, s_or = oracle_roundtrip(img, Q)
            t = gpu(img)
            coef = torch.empty(c_or.size, dtype=torch.int16, device="cuda")
            out = torch.empty_like(t)
            sse = D.dct_codec_fused(plan, [t], quality, coeffs=coef, recon_planes=[out])
            sse_only = D.dct_codec_fused(plan, [t], quality)
            torch.cuda.synchronize()
            assert np.array_equal(coef.cpu().numpy(), c_or)
            assert np.array_equal(out.cpu().numpy(), r_or)
            assert int(sse.cpu()[0]) == s_or
            assert int(sse_only.cpu()[0]) == s_or


def test_custom_tables(D):
    rng = np.random.default_rng(21)
    with D.Plan(512, 512) as plan:
        for k in range(6):
            qt = rng.integers(1, 256, size=64)
            if k == 0:
                qt[:] = 1
            if k == 1:
                qt[:] = 255
            img = rand_img(61, 300, 300 + k)
            c_or, r_or, s_or = oracle_roundtrip(img, qt.reshape(8, 8))
            t = gpu(img)
            coef = D.dct_compress(plan, [t], 0, qtab=qt)
            out = torch.empty_like(t)
            sse = D.dct_reconstruct(plan, coef, [out], 0, qtab=qt, ref_planes=[t])
            torch.cuda.synchronize()
            assert np.array_equal(coef.cpu().numpy(), c_or)
            assert np.array_equal(out.cpu().numpy(), r_or)
            assert int(sse.cpu()[0]) == s_or


def test_yuv420_planes_use_luma_and_chroma_tables(D):
    y, cb, cr = [p.numpy() for p in yuv420_frame(330, 190, seed=5)]
    quality = 75
    with D.Plan(512, 512, layout=D.DCT_LAYOUT_YUV420) as plan:
        ts = [gpu(p) for p in (y, cb, cr)]
        coef = D.dct_compress(plan, ts, quality)
        outs = [torch.empty_like(t) for t in ts]
        sse = D.dct_reconstruct(plan, coef, outs, quality, ref_planes=ts)
        sse_f = D.dct_codec_fused(plan, ts, quality)
        torch.cuda.synchronize()
        off = 0
        got = coef.cpu().numpy()
        for i, p in enumerate((y, cb, cr)):
            Q = ijg.luma_table(quality) if i == 0 else ijg.chroma_table(quality)
            c_or, r_or, s_or = oracle_roundtrip(p, Q)
            assert np.array_equal(got[off:off + c_or.size], c_or)
            off += c_or.size
            assert np.array_equal(outs[i].cpu().numpy(), r_or)
            assert int(sse.cpu()[i]) == s_or
            assert int(sse_f.cpu()[i]) == s_or


def test_pitch_and_unaligned_views(D):
    img = rand_img(45, 77, 33)
    Q = ijg.luma_table(60)
    c_or, r_or, s_or = oracle_roundtrip(img, Q)
    with D.Plan(256, 256) as plan:
        for pitch, off in ((77, 0), (96, 0), (101, 3), (128, 8), (130, 1)):
            buf = torch.zeros(45 * pitch + off + 16, dtype=torch.uint8, device="cuda")
            view = buf[off:off + 45 * pitch].view(45, pitch)[:, :77]
            view.copy_(gpu(img))
            obuf = torch.zeros_like(buf)
            oview = obuf[off:off + 45 * pitch].view(45, pitch)[:, :77]
            coef = D.dct_compress(plan, [view], 60)
            sse = D.dct_reconstruct(plan, coef, [oview], 60, ref_planes=[view])
            torch.cuda.synchronize()
            assert np.array_equal(coef.cpu().numpy(), c_or), (pitch, off)
            assert np.array_equal(oview.cpu().numpy(), r_or), (pitch, off)
            assert int(sse.cpu()[0]) == s_or
            # nothing outside the plane was written
            mask = torch.ones_like(obuf, dtype=torch.bool)
            mask[off:off + 45 * pitch].view(45, pitch)[:, :77] = False
            assert int(obuf[mask].abs().sum()) == 0


def test_psnr_entry_point(D):
    with D.Plan(1024, 1024) as plan:
        for k, (h, w) in enumerate([(1, 1), (7, 13), (64, 64), (99, 1000), (1024, 17)]):
            a = rand_img(h, w, 50 + k)
            b = np.clip(a.astype(int) + np.random.default_rng(k).integers(-20, 21, size=a.shape), 0, 255)
            b = b.astype(np.uint8)
            sse, ps = D.dct_psnr(plan, [gpu(a)], [gpu(b)])
            s_or = psnr.sse(a, b)
            assert int(sse.cpu()[0]) == s_or
            p_or = psnr.psnr_from_sse(s_or, a.size)
            if math.isinf(p_or):
                assert math.isinf(ps[0])
            else:
                assert abs(ps[0] - p_or) <= 1e-9 * abs(p_or)
        # MAX of Eq. 23 read literally as the largest value in O
        a = rand_img(40, 40, 9)
        b = 255 - a
        _, ps = D.dct_psnr(plan, [gpu(a)], [gpu(b)], max_value=float(a.max()))
        assert abs(ps[0] - psnr.psnr(a, b, max_of_original=True)) < 1e-9


def test_statistics_words(D):
    with D.Plan(1024, 1024) as plan:
        for k, (h, w) in enumerate([(8, 8), (37, 29), (256, 264), (300, 517)]):
            img = rand_img(h, w, 70 + k)
            st = torch.zeros(80, dtype=torch.int64, device="cuda")
            D.dct_compress(plan, [gpu(img)], 50, stats=st)
            torch.cuda.synchronize()
            assert st.cpu().tolist() == features.plane_stats(img), (h, w)


@pytest.mark.parametrize("value", [0, 1, 127, 128, 254, 255])
def test_constant_images(D, value):
    img = np.full((24, 40), value, dtype=np.uint8)
    with D.Plan(64, 64) as plan:
        for quality in (1, 50, 100):
            c_or, r_or, s_or = oracle_roundtrip(img, ijg.luma_table(quality))
            t = gpu(img)
            coef = D.dct_compress(plan, [t], quality)
            out = torch.empty_like(t)
            sse = D.dct_reconstruct(plan, coef, [out], quality, ref_planes=[t])
            torch.cuda.synchronize()
            assert np.array_equal(coef.cpu().numpy(), c_or)
            assert np.array_equal(out.cpu().numpy(), r_or)
            assert int(sse.cpu()[0]) == s_or


def test_checkerboard_extremes(D):
    i, j = np.mgrid[0:64, 0:64]
    img = np.where((i + j) % 2 == 0, 255, 0).astype(np.uint8)
    for quality in (1, 100):
        c_or, r_or, s_or = oracle_roundtrip(img, ijg.luma_table(quality))
        with D.Plan(64, 64) as plan:
            t = gpu(img)
            coef = D.dct_compress(plan, [t], quality)
            out = torch.empty_like(t)
            sse = D.dct_reconstruct(plan, coef, [out], quality, ref_planes=[t])
            torch.cuda.synchronize()
            assert np.array_equal(coef.cpu().numpy(), c_or)
            assert np.array_equal(out.cpu().numpy(), r_or)
            assert int(sse.cpu()[0]) == s_or


def test_reconstruct_of_arbitrary_int16_is_defined(D):
    # the dequantiser clamp gives defined output for any int16 input
    rng = np.random.default_rng(3)
    c = rng.integers(-32768, 32768, size=(5, 7, 8, 8)).astype(np.int16)
    Q = ijg.luma_table(30)
    r_or = codec.reconstruct_plane(c, Q, 40, 56)
    with D.Plan(64, 64) as plan:
        out = torch.empty(40, 56, dtype=torch.uint8, device="cuda")
        D.dct_reconstruct(plan, gpu(c.reshape(-1)), [out], 30)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), r_or)


def test_invalid_arguments_enqueue_nothing(D):
    t = torch.zeros(16, 16, dtype=torch.uint8, device="cuda")
    with D.Plan(32, 32) as plan:
        coef = torch.zeros(4 * 64 + 8, dtype=torch.int16, device="cuda")
        for kw in (dict(quality=101), dict(quality=-3), dict(quality=0)):
            with pytest.raises(D.DctError) as ei:
                D.dct_compress(plan, [t], kw["quality"], coeffs=coef)
            assert ei.value.status == 1
        with pytest.raises(D.DctError):   # larger than the plan
            D.dct_compress(plan, [torch.zeros(40, 16, dtype=torch.uint8, device="cuda")], 50)
        with pytest.raises(D.DctError):   # misaligned coefficient buffer
            D.dct_compress(plan, [t], 50, coeffs=coef[1:])
        with pytest.raises(D.DctError):   # five planes
            D.dct_compress(plan, [t] * 5, 50)
        with pytest.raises(D.DctError):   # ref without sse / size mismatch
            D.dct_reconstruct(plan, coef, [t], 50, ref_planes=[torch.zeros(8, 16, dtype=torch.uint8,
                                                                           device="cuda")])
        torch.cuda.synchronize()
        assert int(coef.abs().sum()) == 0
    with pytest.raises(D.DctError):
        D.Plan(0, 10)


def test_full_size_workload_sampled(D):
    """8192 x 8192 grey plus a 3840 x 2160 4:2:0 frame at quality 75 through
    the direct plane calls (dct_compress, dct_reconstruct): sampled blocks
    against the oracle, the SSE against the reconstruction it belongs to.
    The batched configuration the benchmark times is tested in
    test_gpu_batch.py."""
    dev = "cuda"
    grey = powerlaw_image(8192, 8192, seed=11, device=dev)
    y, cb, cr = yuv420_frame(3840, 2160, seed=12, device=dev)
    quality = 75
    rng = np.random.default_rng(0)
    with D.Plan(8192, 8192, layout=D.DCT_LAYOUT_YUV420) as plan_yuv, D.Plan(8192, 8192) as plan_g:
        for plan, planes in ((plan_g, [grey]), (plan_yuv, [y, cb, cr])):
            coef = D.dct_compress(plan, planes, quality)
            outs = [torch.empty_like(p) for p in planes]
            sse = D.dct_reconstruct(plan, coef, outs, quality, ref_planes=planes)
            torch.cuda.synchronize()
            off = 0
            for i, p in enumerate(planes):
                h, w = p.shape
                nby, nbx = (h + 7) // 8, (w + 7) // 8
                Q = ijg.luma_table(quality) if (i == 0 or plan is plan_g) else ijg.chroma_table(quality)
                # 2048 random blocks plus the last block row and column
                bys = np.concatenate([rng.integers(0, nby, 2048), np.full(nbx, nby - 1), np.arange(nby)])
                bxs = np.concatenate([rng.integers(0, nbx, 2048), np.arange(nbx), np.full(nby, nbx - 1)])
                sel = np.unique(bys * nbx + bxs)
                host = p.cpu().numpy()
                blocks = codec.plane_to_blocks(host).reshape(-1, 8, 8)[sel]
                c_or = codec.compress_blocks(blocks, Q)
                got = coef[off:off + nby * nbx * 64].view(-1, 8, 8)[torch.from_numpy(sel).cuda()].cpu().numpy()
                assert np.array_equal(got, c_or)
                r_or = codec.reconstruct_blocks(c_or, Q)
                rec = codec.plane_to_blocks(outs[i].cpu().numpy()).reshape(-1, 8, 8)[sel]
                by_s, bx_s = sel // nbx, sel % nbx
                for k in range(sel.size):   # compare the in-plane part of each sampled block
                    nr = min(8, h - 8 * by_s[k])
                    nc = min(8, w - 8 * bx_s[k])
                    assert np.array_equal(rec[k, :nr, :nc], r_or[k, :nr, :nc])
                d = outs[i].to(torch.int64) - p.to(torch.int64)
                assert int(sse.cpu()[i]) == int((d * d).sum())
                off += nby * nbx * 64

"""RGB input fused into the forward path (dct_compress_rgb) against the
oracle route: RGB -> YCbCr 4:2:0 (oracle/color.py), then the forward path
of Sec. 2.5.2 / 3.2 on each plane (luminance table for Y, chrominance for
Cb and Cr), bit for bit; and against the library's own two-kernel route."""
import numpy as np
import pytest
import torch

from oracle import codec, color, ijg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def oracle_codes(rgb, quality=None, qtab=None):
    y, cb, cr = color.rgb_to_yuv420(rgb)
    if qtab is None:
        ql, qc = ijg.luma_table(quality), ijg.chroma_table(quality)
    else:
        t = np.asarray(qtab, dtype=np.int64).reshape(-1, 8, 8)
        ql, qc = t[0], t[-1]
    return np.concatenate([codec.compress_plane(y, ql).reshape(-1), codec.compress_plane(cb, qc).reshape(-1),
                           codec.compress_plane(cr, qc).reshape(-1)])


def rgb_image(h, w, seed):
    """Smooth colour content plus noise and a hard edge (so both chroma
    planes carry structure)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w]
    base = np.stack([128 + 100 * np.sin(xx / 7.0 + k) * np.cos(yy / 11.0 - k) for k in range(3)], axis=-1)
    base += rng.normal(0, 12, size=base.shape)
    base[:, w // 3:] += np.array([60, -40, 20])
    return np.clip(np.rint(base), 0, 255).astype(np.uint8)


SHAPES = [(1, 1), (1, 7), (5, 1), (8, 8), (13, 29), (16, 16), (17, 33), (31, 47), (40, 520), (33, 530),
          (135, 241), (250, 300), (720, 1280)]


@pytest.mark.parametrize("h,w", SHAPES)
def test_fused_rgb_codes_match_the_oracle(D, h, w):
    rgb = rgb_image(h, w, h * 7 + w)
    q = [10, 35, 50, 75, 90, 100][(h + w) % 6]
    with D.Plan(2048, 2048) as plan:
        codes = D.dct_compress_rgb(plan, torch.from_numpy(rgb).cuda(), q)
        torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy(), oracle_codes(rgb, q)), (h, w, q)


def test_fused_rgb_custom_tables_pitch_and_unaligned_view(D):
    h, w = 77, 301
    rgb = rgb_image(h, w, 3)
    rng = np.random.default_rng(4)
    tabs = rng.integers(1, 256, size=128).astype(np.uint16)
    # rows padded to 3 * 320 bytes and the frame starting 5 bytes into the buffer
    buf = torch.zeros(5 + h * 960, dtype=torch.uint8, device="cuda")
    view = torch.as_strided(buf, (h, w, 3), (960, 3, 1), storage_offset=5)
    view.copy_(torch.from_numpy(rgb))
    with D.Plan(512, 512) as plan:
        codes = D.dct_compress_rgb(plan, view, 0, qtab=tabs)
        one = D.dct_compress_rgb(plan, view, 0, qtab=tabs[:64])
        torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy(), oracle_codes(rgb, qtab=tabs))
    assert np.array_equal(one.cpu().numpy(), oracle_codes(rgb, qtab=tabs[:64]))
    assert int(buf[:5].abs().sum()) == 0


def test_fused_rgb_equals_the_two_kernel_route(D):
    h, w = 1080, 1920
    rgb = torch.from_numpy(rgb_image(h, w, 9)).cuda()
    with D.Plan(1920, 1080, layout=D.DCT_LAYOUT_YUV420) as plan:
        fused = D.dct_compress_rgb(plan, rgb, 75)
        y, cb, cr = D.dct_rgb_to_yuv420(rgb)
        two = D.dct_compress(plan, [y, cb, cr], 75)
        torch.cuda.synchronize()
    assert torch.equal(fused, two)


def test_fused_rgb_rejects_bad_arguments(D):
    rgb = torch.zeros(16, 16, 3, dtype=torch.uint8, device="cuda")
    with D.Plan(8, 8) as plan:
        with pytest.raises(D.DctError):
            D.dct_compress_rgb(plan, rgb, 50)                 # larger than the plan allows
    with D.Plan(64, 64) as plan:
        with pytest.raises(D.DctError):
            D.dct_compress_rgb(plan, rgb, 101)
        bad = torch.zeros(D.rgb_coeff_count(16, 16) + 8, dtype=torch.int16, device="cuda")[1:]
        with pytest.raises(D.DctError):
            D.dct_compress_rgb(plan, rgb, 50, coeffs=bad)     # not 16-byte aligned

"""GPU parity of RGB -> YCbCr 4:2:0 against the oracle, and a colour frame
through the codec."""
import numpy as np
import pytest
import torch

from oracle import codec, color, ijg, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


@pytest.mark.parametrize("h,w", [(1, 1), (1, 7), (5, 1), (8, 8), (13, 29), (64, 96), (135, 241), (720, 1280)])
def test_rgb_to_yuv420_bit_exact(D, h, w):
    rng = np.random.default_rng(h * 1000 + w)
    rgb = rng.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    y, cb, cr = D.dct_rgb_to_yuv420(torch.from_numpy(rgb).cuda())
    torch.cuda.synchronize()
    ry, rb, rr = color.rgb_to_yuv420(rgb)
    assert np.array_equal(y.cpu().numpy(), ry)
    assert np.array_equal(cb.cpu().numpy(), rb)
    assert np.array_equal(cr.cpu().numpy(), rr)


def test_padded_rgb_rows(D):
    rng = np.random.default_rng(3)
    buf = torch.from_numpy(rng.integers(0, 256, size=(40, 70, 3)).astype(np.uint8)).cuda()
    view = buf[:, :61, :]                      # row pitch 210 bytes, width 61
    y, cb, cr = D.dct_rgb_to_yuv420(view)
    ry, rb, rr = color.rgb_to_yuv420(view.cpu().numpy())
    assert np.array_equal(y.cpu().numpy(), ry) and np.array_equal(cb.cpu().numpy(), rb)
    assert np.array_equal(cr.cpu().numpy(), rr)


def test_colour_frame_through_the_codec(D):
    from synth import powerlaw_image
    r, g, b = (powerlaw_image(96, 128, seed=s).numpy() for s in (1, 2, 3))
    rgb = np.stack([r, g, b], axis=-1)
    y, cb, cr = D.dct_rgb_to_yuv420(torch.from_numpy(rgb).cuda())
    with D.Plan(128, 96, layout=D.DCT_LAYOUT_YUV420) as plan:
        sse = D.dct_codec_fused(plan, [y, cb, cr], 80)
        torch.cuda.synchronize()
    for i, p in enumerate(color.rgb_to_yuv420(rgb)):
        Q = ijg.luma_table(80) if i == 0 else ijg.chroma_table(80)
        rec = codec.reconstruct_plane(codec.compress_plane(p, Q), Q, *p.shape)
        assert int(sse[i]) == psnr.sse(p, rec)


def test_rgb_invalid_sizes(D):
    rgb = torch.zeros(8, 8, 3, dtype=torch.uint8, device="cuda")
    with pytest.raises(D.DctError):
        D.dct_rgb_to_yuv420(rgb, cb=torch.zeros(3, 4, dtype=torch.uint8, device="cuda"))

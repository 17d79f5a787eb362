"""Exact rounding ties of the quantiser, through every kernel family.

The kernels drop the sign term of the quantiser everywhere except the four
entries (u, v in {0, 4}) whose multiplier can be a high power of two.  Those
four outputs are sums of samples only (no CORDIC rotation reaches them), so
a block with one sample at 128 + d gives Y00, Y04, Y40 and Y44 all equal to
+-16 d; with a flat table Q = 2^j (M = 2^(25-j)) an exact tie needs
|16 d| = 2^(6+j) * odd.  The image below places such spikes of both signs
at every position of a block; the GPU results must equal the oracle's."""
import numpy as np
import pytest
import torch

from oracle import codec, ijg, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def spike_image(j):
    d = 4 << j                                   # |16 d| = 2^(6 + j): a tie for Q = 2^j
    deltas = [d, -d, 3 * d, -3 * d]
    deltas = [x for x in deltas if 0 <= 128 + x <= 255]
    blocks = []
    for x in deltas:
        for pos in range(64):
            b = np.full(64, 128, dtype=np.int64)
            b[pos] = 128 + x
            blocks.append(b.reshape(8, 8))
    nb = len(blocks)
    cols = 16
    rows = (nb + cols - 1) // cols
    img = np.full((rows * 8, cols * 8), 128, dtype=np.uint8)
    for k, b in enumerate(blocks):
        r, c = divmod(k, cols)
        img[8 * r:8 * r + 8, 8 * c:8 * c + 8] = b
    return img


def oracle(img, Q):
    c = codec.compress_plane(img, Q)
    r = codec.reconstruct_plane(c, Q, *img.shape)
    return c.reshape(-1), r, psnr.sse(img, r)


@pytest.mark.parametrize("j", [0, 1, 2, 3, 4])
def test_ties_all_kernel_families(D, j):
    img = spike_image(j)
    qtab = np.full(64, 1 << j, dtype=np.uint16)
    c_or, r_or, s_or = oracle(img, qtab.reshape(8, 8).astype(np.int64))
    # the spikes do land on exact ties at the four sign-aware entries
    m = codec.quant_multipliers(qtab.reshape(8, 8))
    assert int(m[0, 0]) == 1 << (25 - j)
    t = torch.from_numpy(img).cuda()
    h, w = img.shape
    with D.Plan(w, h, max_batch=1) as plan:
        coef = D.dct_compress(plan, [t], 0, qtab=qtab)
        out = torch.empty_like(t)
        sse = D.dct_reconstruct(plan, coef, [out], 0, qtab=qtab, ref_planes=[t])
        coef_f = torch.empty_like(coef)
        rec_f = torch.empty_like(t)
        sse_f = D.dct_codec_fused(plan, [t], 0, qtab=qtab, coeffs=coef_f, recon_planes=[rec_f])
        torch.cuda.synchronize()
        assert np.array_equal(coef.cpu().numpy(), c_or)
        assert np.array_equal(out.cpu().numpy(), r_or)
        assert int(sse[0]) == s_or
        assert np.array_equal(coef_f.cpu().numpy(), c_or)
        assert np.array_equal(rec_f.cpu().numpy(), r_or)
        assert int(sse_f[0]) == s_or
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        for lanes in (1, 2):
            cb = torch.zeros_like(coef)
            rb = torch.zeros_like(t)
            sb = torch.zeros(1, dtype=torch.int64, device="cuda")
            arr = D.make_batch_items([t], [0], coeffs=[cb], recons=[rb], qtabs=[qtab])
            D.dct_batch_prepare(plan, arr, C | R | S, sse=sb, shape=(128, 2, 32, lanes))
            D.dct_batch_launch(plan)
            torch.cuda.synchronize()
            assert np.array_equal(cb.cpu().numpy(), c_or), lanes
            assert np.array_equal(rb.cpu().numpy(), r_or), lanes
            assert int(sb[0]) == s_or, lanes

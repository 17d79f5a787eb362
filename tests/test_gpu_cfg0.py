"""The plain method's small configuration, exactly as the benchmark's cfg0
line runs it: one 512 x 512 grey image of 8 random 2-D sinusoids plus
Gaussian noise (seed 0, generated on the GPU), IJG luminance table at
quality 50 (the quantiser of Sec. 3.2), compared element by element with the
CPU oracle: coefficients, reconstruction and the SSE of Eq. 24, through the
direct calls and the one-item batch graph."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_cfg0_image_bit_exact_against_the_oracle(cuda_ok):
    from oracle import codec, ijg, psnr
    from paper_1306_1373_gb300 import dctgb as D
    from synth import sinusoid_image
    img = sinusoid_image(512, 512, seed=0, device="cuda")
    host = img.cpu().numpy()
    Q = ijg.luma_table(50)
    c_or = codec.compress_plane(host, Q)
    r_or = codec.reconstruct_plane(c_or, Q, 512, 512)
    s_or = psnr.sse(host, r_or)
    with D.Plan(512, 512, max_batch=1) as plan:
        coef = D.dct_compress(plan, [img], 50)
        rec = torch.empty_like(img)
        sse = D.dct_reconstruct(plan, coef, [rec], 50, ref_planes=[img])
        coef_f = torch.empty_like(coef)
        rec_f = torch.empty_like(img)
        sse_f = D.dct_codec_fused(plan, [img], 50, coeffs=coef_f, recon_planes=[rec_f])
        coef_b = torch.empty_like(coef)
        rec_b = torch.empty_like(img)
        sse_b = torch.zeros(1, dtype=torch.int64, device="cuda")
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        D.dct_batch_prepare(plan, D.make_batch_items([img], [50], coeffs=[coef_b], recons=[rec_b]), C | R | S,
                            sse=sse_b)
        D.dct_batch_launch(plan)
        D.dct_batch_launch(plan)
        torch.cuda.synchronize()
    for c in (coef, coef_f, coef_b):
        assert np.array_equal(c.cpu().numpy(), c_or.reshape(-1))
    for r in (rec, rec_f, rec_b):
        assert np.array_equal(r.cpu().numpy(), r_or)
    for s in (sse, sse_f, sse_b):
        assert int(s[0]) == s_or
    p = D.dct_psnr_from_sse(s_or, 512 * 512)
    assert abs(p - psnr.psnr_from_sse(s_or, 512 * 512)) <= 1e-9 * p

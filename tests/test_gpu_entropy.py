"""GPU parity of the rate statistics (symbol counts, amplitude bits) against
the oracle, and the bits they imply."""
import numpy as np
import pytest
import torch

from oracle import codec, entropy, ijg
from synth import powerlaw_image, yuv420_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


@pytest.mark.parametrize("quality", [5, 50, 95, 100])
def test_symbol_statistics_match_oracle(D, quality):
    with D.Plan(1024, 1024) as plan:
        for k, (h, w) in enumerate([(8, 8), (37, 29), (256, 264), (300, 517)]):
            img = powerlaw_image(h, w, seed=quality * 10 + k).numpy()
            t = torch.from_numpy(img).cuda()
            coef = D.dct_compress(plan, [t], quality)
            st = D.dct_entropy_stats(plan, coef, [(h, w)]).cpu().numpy()[0]
            ref = codec.compress_plane(img, ijg.luma_table(quality)).reshape(-1, 64)
            dc, ac, amp, nb = entropy.plane_histograms(ref)
            assert st[:16].tolist() == dc and st[16:272].tolist() == ac
            assert int(st[272]) == amp and int(st[273]) == nb
            assert abs(D.dct_entropy_bits(st) - entropy.plane_bits(ref)) <= 1e-9 * max(1.0, entropy.plane_bits(ref))
            assert D.dct_huffman_bits(st) == entropy.plane_huffman_bits(ref)
            assert D.dct_huffman_bits(st) >= D.dct_entropy_bits(st) - 1e-6


def test_yuv420_statistics_and_rate_falls_with_quality(D):
    planes = [p.cuda() for p in yuv420_frame(320, 240, seed=7)]
    shapes = [tuple(p.shape) for p in planes]
    bits = []
    with D.Plan(320, 240, layout=D.DCT_LAYOUT_YUV420) as plan:
        for quality in (90, 50, 10):
            coef = D.dct_compress(plan, planes, quality)
            st = D.dct_entropy_stats(plan, coef, shapes).cpu().numpy()
            bits.append(sum(D.dct_entropy_bits(r) for r in st))
            off = 0
            for i, p in enumerate(planes):
                Q = ijg.luma_table(quality) if i == 0 else ijg.chroma_table(quality)
                ref = codec.compress_plane(p.cpu().numpy(), Q).reshape(-1, 64)
                dc, ac, amp, nb = entropy.plane_histograms(ref)
                assert st[i, :16].tolist() == dc and st[i, 16:272].tolist() == ac and int(st[i, 272]) == amp
    assert bits[0] > bits[1] > bits[2] > 0

"""The forward kernels' float micro-rotations at the forward graph's extreme
nodes: blocks holding the sign pattern of every 2-D cosine basis (0 and
255 on the two signs, and the reverse), which drive the transform's
outputs towards their interval bounds, plus checkerboards, edges and
constant blocks, through every forward-only entry (direct compress, the
batched forward pass in both tile layouts, the statistics pass) and the
two-pass graph (whose inverse kernel reads its own codes without the
dequantiser clamp) at N = 4, 5 and 6, against the oracle bit for bit
(Sec. 2.5.2)."""
import numpy as np
import pytest
import torch

from oracle import codec, ijg

pytestmark = pytest.mark.gpu
NS = (4, 5, 6)


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def extreme_image():
    ii, jj = np.mgrid[0:8, 0:8]
    blocks = []
    for u in range(8):
        for v in range(8):
            basis = np.cos((2 * ii + 1) * u * np.pi / 16) * np.cos((2 * jj + 1) * v * np.pi / 16)
            blocks.append(np.where(basis >= 0, 255, 0))
            blocks.append(np.where(basis >= 0, 0, 255))
    blocks += [np.where((ii + jj) % 2, 255, 0), np.where((ii + jj) % 2, 0, 255), np.where(jj < 4, 0, 255),
               np.where(ii < 4, 255, 0), np.full((8, 8), 0), np.full((8, 8), 255), np.full((8, 8), 128)]
    cols = 16
    rows = (len(blocks) + cols - 1) // cols
    img = np.full((rows * 8, cols * 8), 128, dtype=np.uint8)
    for k, b in enumerate(blocks):
        r, c = divmod(k, cols)
        img[8 * r:8 * r + 8, 8 * c:8 * c + 8] = b
    return img


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("quality", [1, 50, 100])
def test_forward_entries_at_extreme_nodes(D, n, quality):
    img = extreme_image()
    Q = ijg.luma_table(quality)
    want = codec.compress_plane(img, Q, n).reshape(-1)
    t = torch.from_numpy(img).cuda()
    with D.cordic_variant(n):
        with D.Plan(img.shape[1], img.shape[0], max_batch=2) as plan:
            direct = D.dct_compress(plan, [t], quality)
            got = {"direct": direct}
            for lanes in (1, 2):
                coef = torch.zeros(want.size, dtype=torch.int16, device="cuda")
                D.dct_batch_prepare(plan, D.make_batch_items([t], [quality], coeffs=[coef]), D.DCT_OP_COMPRESS,
                                    shape=(128, 4, 32, lanes))
                D.dct_batch_launch(plan)
                got["batch%d" % lanes] = coef
            st = torch.zeros(80, dtype=torch.int64, device="cuda")
            got["stats_pass"] = D.dct_compress(plan, [t], quality, stats=st)
            torch.cuda.synchronize()
    for k, v in got.items():
        assert np.array_equal(v.cpu().numpy(), want), (n, quality, k)
    # band energies of the unquantised forward output
    y = codec.forward_coefficients(codec.plane_to_blocks(img).reshape(-1, 8, 8), n)
    band = ((np.abs(y) >> 5) ** 2).sum(axis=0).reshape(-1)
    assert np.array_equal(st.cpu().numpy()[:64], band)


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("quality", [1, 50, 100])
@pytest.mark.parametrize("lanes", [1, 2])
def test_two_pass_inverse_on_own_codes_at_extremes(D, n, quality, lanes):
    """The two-pass graph's inverse kernel dequantises the codes its forward
    kernel wrote without the clamp (|q Q| stays far inside 4096); at the
    extreme blocks and the coarsest and finest tables its reconstruction and
    SSE equal the oracle's clamped definition."""
    from oracle import psnr
    img = extreme_image()
    Q = ijg.luma_table(quality)
    c_or = codec.compress_plane(img, Q, n)
    r_or = codec.reconstruct_plane(c_or, Q, *img.shape, n=n)
    t = torch.from_numpy(img).cuda()
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    with D.cordic_variant(n):
        with D.Plan(img.shape[1], img.shape[0], max_batch=2) as plan:
            coef = torch.zeros(c_or.size, dtype=torch.int16, device="cuda")
            rec = torch.zeros_like(t)
            sse = torch.zeros(1, dtype=torch.int64, device="cuda")
            D.dct_batch_prepare(plan, D.make_batch_items([t], [quality], coeffs=[coef], recons=[rec]), C | R | S | T,
                                sse=sse, shape=(128, 4, 32, lanes))
            D.dct_batch_launch(plan)
            torch.cuda.synchronize()
    assert np.array_equal(coef.cpu().numpy(), c_or.reshape(-1))
    assert np.array_equal(rec.cpu().numpy(), r_or)
    assert int(sse[0]) == psnr.sse(img, r_or)

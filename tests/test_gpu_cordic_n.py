"""GPU parity of the libraries built at other CORDIC iteration counts
(N = 4 and 5; Sec. 2.5.2 gives no count, the spec file's default is 6):
every kernel family against the oracle run at the same N, bit for bit, on
ragged planes, uneven batches in both tile layouts, exact quantiser ties
and the rate controller's statistics words."""
import numpy as np
import pytest
import torch

from oracle import codec, features, ijg, psnr
from synth import powerlaw_image, sinusoid_image

pytestmark = pytest.mark.gpu
NS = (4, 5)


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def oracle(img, Q, n):
    c = codec.compress_plane(img, Q, n)
    r = codec.reconstruct_plane(c, Q, *img.shape, n=n)
    return c.reshape(-1), r, psnr.sse(img, r)


@pytest.mark.parametrize("n", NS)
def test_direct_calls_match_the_oracle_at_n(D, n):
    shapes = [(1, 1), (8, 8), (13, 7), (37, 130), (96, 64), (250, 77)]
    with D.cordic_variant(n):
        assert D.dct_spec_query()["N"] == n
        with D.Plan(256, 256) as plan:
            for k, (h, w) in enumerate(shapes):
                img = powerlaw_image(h, w, seed=300 + k, device="cuda")
                host = img.cpu().numpy()
                q = (10, 50, 75, 95, 100, 1)[k]
                Q = ijg.luma_table(q)
                c_or, r_or, s_or = oracle(host, Q, n)
                coef = D.dct_compress(plan, [img], q)
                rec = torch.empty_like(img)
                sse = D.dct_reconstruct(plan, coef, [rec], q, ref_planes=[img])
                coef_f = torch.empty_like(coef)
                rec_f = torch.empty_like(img)
                sse_f = D.dct_codec_fused(plan, [img], q, coeffs=coef_f, recon_planes=[rec_f])
                torch.cuda.synchronize()
                assert np.array_equal(coef.cpu().numpy(), c_or), (n, h, w)
                assert np.array_equal(coef_f.cpu().numpy(), c_or), (n, h, w)
                assert np.array_equal(rec.cpu().numpy(), r_or), (n, h, w)
                assert np.array_equal(rec_f.cpu().numpy(), r_or), (n, h, w)
                assert int(sse[0]) == s_or and int(sse_f[0]) == s_or, (n, h, w)


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("ops_name", ["fused", "two_pass", "compress"])
@pytest.mark.parametrize("lanes", [1, 2])
def test_batches_match_the_oracle_at_n(D, n, ops_name, lanes):
    rng = np.random.default_rng(40 + n)
    srcs, quals, chroma = [], [], []
    for i in range(9):
        h, w = int(rng.integers(8, 200)), int(rng.integers(8, 200))
        srcs.append(powerlaw_image(h, w, seed=700 + i, beta=float(rng.uniform(1, 3)), device="cuda"))
        quals.append(int(rng.integers(5, 101)))
        chroma.append(bool(i % 2))
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    ops = {"fused": C | R | S, "two_pass": C | R | S | T, "compress": C}[ops_name]
    with D.cordic_variant(n):
        coefs = [torch.zeros(D.coeff_count([s.shape]), dtype=torch.int16, device="cuda") for s in srcs]
        recs = [torch.zeros_like(s) for s in srcs]
        sse = torch.zeros(len(srcs), dtype=torch.int64, device="cuda")
        with D.Plan(256, 256, max_batch=16) as plan:
            D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs, chroma=chroma), ops,
                                sse=sse if ops & S else None, shape=(128, 4, 32, lanes))
            D.dct_batch_launch(plan)
            D.dct_batch_launch(plan)
            torch.cuda.synchronize()
    for i, s in enumerate(srcs):
        host = s.cpu().numpy()
        Q = ijg.chroma_table(quals[i]) if chroma[i] else ijg.luma_table(quals[i])
        c_or, r_or, s_or = oracle(host, Q, n)
        assert np.array_equal(coefs[i].cpu().numpy(), c_or), i
        if ops & R:
            assert np.array_equal(recs[i].cpu().numpy(), r_or), i
        if ops & S:
            assert int(sse[i]) == s_or, i


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("j", [0, 2, 4])
def test_exact_ties_at_n(D, n, j):
    """One-sample spikes put Y00, Y04, Y40 and Y44 (sums of samples only, at
    every N) on exact rounding ties of a flat table Q = 2^j."""
    d = 4 << j
    blocks = []
    for x in (d, -d, 3 * d, -3 * d):
        if 0 <= 128 + x <= 255:
            for pos in range(64):
                b = np.full(64, 128, dtype=np.uint8)
                b[pos] = 128 + x
                blocks.append(b.reshape(8, 8))
    cols = 16
    rows = (len(blocks) + cols - 1) // cols
    img = np.full((rows * 8, cols * 8), 128, dtype=np.uint8)
    for k, b in enumerate(blocks):
        r, c = divmod(k, cols)
        img[8 * r:8 * r + 8, 8 * c:8 * c + 8] = b
    qtab = np.full(64, 1 << j, dtype=np.uint16)
    c_or, r_or, s_or = oracle(img, qtab.reshape(8, 8).astype(np.int64), n)
    t = torch.from_numpy(img).cuda()
    with D.cordic_variant(n):
        with D.Plan(img.shape[1], img.shape[0]) as plan:
            coef_f = torch.empty(c_or.size, dtype=torch.int16, device="cuda")
            rec_f = torch.empty_like(t)
            sse_f = D.dct_codec_fused(plan, [t], 0, qtab=qtab, coeffs=coef_f, recon_planes=[rec_f])
            coef = D.dct_compress(plan, [t], 0, qtab=qtab)
            torch.cuda.synchronize()
    assert np.array_equal(coef_f.cpu().numpy(), c_or) and np.array_equal(coef.cpu().numpy(), c_or)
    assert np.array_equal(rec_f.cpu().numpy(), r_or) and int(sse_f[0]) == s_or


@pytest.mark.parametrize("n", NS)
def test_statistics_words_at_n(D, n):
    """The statistics pass (band energies of the unquantised forward output)
    against the oracle's words at the same N."""
    img = sinusoid_image(72, 104, seed=5, device="cuda")
    with D.cordic_variant(n):
        with D.Plan(128, 128) as plan:
            st = torch.zeros(80, dtype=torch.int64, device="cuda")
            D.dct_compress(plan, [img], 50, stats=st)
            torch.cuda.synchronize()
    host = img.cpu().numpy()
    blocks = codec.plane_to_blocks(host).reshape(-1, 8, 8)
    y = codec.forward_coefficients(blocks, n)
    e = (np.abs(y) >> 5) ** 2
    band = e.sum(axis=0).reshape(-1)
    got = st.cpu().numpy().astype(np.uint64)
    assert np.array_equal(got[:64].astype(np.int64), band)
    ref = features.plane_stats(host)                      # pixel words do not depend on N
    assert list(got[64:78].astype(np.int64)[:8]) == ref[64:72]

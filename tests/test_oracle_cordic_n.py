"""The fixed-point reading at every CORDIC iteration count the library is
built for (N = 4, 5 and the spec's 6; Sec. 2.5.2 gives no count): every
proof the kernels rely on is re-run at each N with the oracle's own tables
and bounds, and the variant libraries' host tables equal the oracle's."""
import numpy as np
import pytest

from oracle import codec, exact_dct, ijg, interval, linear, psnr, spec
from oracle.cordic_loeffler import Sigmas, cordic_gain, gains

NS = (4, 5, 6)
TIE_ENTRIES = {(0, 0), (0, 4), (4, 0), (4, 4)}


def trailing_zeros(m):
    m = int(m)
    return (m & -m).bit_length() - 1


@pytest.mark.parametrize("n", NS)
def test_word_widths_at_every_n(n):
    sig = Sigmas(n)
    f_row, f_col, _ = interval.forward_bounds(sig=sig)
    i_col, i_row = interval.inverse_bounds(n=n)
    i_col2, i_row2 = interval.inverse_bounds(dc_offset=(1 << (spec.R + 2)) + (128 << (spec.R + 3)), n=n)
    assert max(f_row, f_col, i_col, i_row, i_col2, i_row2) < 2 ** 31
    # the tie-free quantiser argument needs |Y| < 2^20, and the clamp-free
    # dequantiser q * (Q W) of the fused kernels and of the two-pass inverse
    # (which reads back its own graph's codes) needs |q Q| within the 4096 clamp
    assert f_col < 2 ** 20
    bits, _ = interval.worst_case_product_bits(f_col, n=n)
    assert bits <= 63
    bound = linear.cordic_vs_exact_bound(n).max()
    assert 1024 + bound + 255 / 2 + 1 < spec.DQ_CLAMP


@pytest.mark.parametrize("n", NS)
def test_quantiser_tie_freeness_at_every_n(n):
    for q in range(1, 256):
        m = codec.quant_multipliers(np.full(64, q), n)
        for u in range(8):
            for v in range(8):
                if (u, v) not in TIE_ENTRIES:
                    assert trailing_zeros(m[u, v]) <= 11, (n, u, v, q)


@pytest.mark.parametrize("n", NS)
def test_error_bound_holds_at_every_n(n):
    bound = linear.cordic_vs_exact_bound(n)
    rng = np.random.default_rng(10 + n)
    b = rng.integers(0, 256, size=(3000, 8, 8)).astype(np.uint8)
    y = codec.forward_coefficients(b, n).astype(np.float64)
    g = np.array(gains(n))
    xs = y / (8.0 * (1 << spec.P) * np.outer(g, g))
    xe = exact_dct.dct2(b.astype(np.float64) - 128.0)
    assert (np.abs(xs - xe) <= bound + 1e-9).all()


def test_fewer_iterations_move_further_from_the_exact_dct():
    """The bound and the observed error grow as N falls; the gains follow
    the closed form K_N = prod sqrt(1 + 4^-i)."""
    bounds = [linear.cordic_vs_exact_bound(n).max() for n in NS]
    assert bounds[0] > bounds[1] > bounds[2]
    for n in NS:
        k = 1.0
        for i in range(1, n + 1):
            k *= (1.0 + 4.0 ** -i) ** 0.5
        assert abs(cordic_gain(n) - k) < 1e-15


@pytest.mark.parametrize("n", NS)
def test_round_trip_and_table3_claim_at_every_n(n):
    """Quality 100 reconstructs within 2 levels; at quality 50 the Cordic
    pipeline's PSNR stays below the exact DCT's plus 0.05 dB (the direction
    Tables 3-4 report)."""
    from synth import sinusoid_image
    rng = np.random.default_rng(6)
    b = rng.integers(0, 256, size=(2000, 8, 8)).astype(np.uint8)
    Q = ijg.luma_table(100)
    r = codec.reconstruct_blocks(codec.compress_blocks(b, Q, n), Q, n)
    assert np.abs(r.astype(int) - b.astype(int)).max() <= 2
    img = sinusoid_image(128, 128, seed=0).numpy()
    Q = ijg.luma_table(50)
    rc = codec.reconstruct_plane(codec.compress_plane(img, Q, n), Q, 128, 128, n)
    blocks = codec.plane_to_blocks(img).reshape(-1, 8, 8)
    re = exact_dct.exact_reconstruct_blocks(exact_dct.exact_compress_blocks(blocks, Q), Q)
    re = codec.blocks_to_plane(re.reshape(16, 16, 8, 8), 128, 128)
    assert psnr.psnr_from_sse(psnr.sse(img, rc), img.size) <= psnr.psnr_from_sse(psnr.sse(img, re), img.size) + 0.05


@pytest.mark.parametrize("n", (4, 5))
def test_variant_library_reports_its_n_and_the_oracle_tables(n):
    from paper_1306_1373_gb300 import dctgb as D
    with D.cordic_variant(n):
        info = D.dct_spec_query()
        assert info["N"] == n
        s = Sigmas(n)
        mask = lambda sig: sum(1 << i for i, v in enumerate(sig, start=1) if v > 0)
        assert (info["sigma_odd_upper"], info["sigma_odd_lower"], info["sigma_even"]) == \
            (mask(s.odd_upper), mask(s.odd_lower), mask(s.even))
        w = codec.dequant_weights(n)
        for chroma in (0, 1):
            for q in range(1, 101):
                Qt, M, W = D.dct_tables(q, chroma=chroma)
                q_or = ijg.chroma_table(q) if chroma else ijg.luma_table(q)
                assert (M == codec.quant_multipliers(q_or, n)).all() and (W == w).all(), (n, q)
    assert D.dct_spec_query()["N"] == spec.N

"""Pins for the fixed-point Cordic-Loeffler oracle (Sec. 2.5.2, Fig. 1).

Each pin ties the oracle to something outside itself: the textbook DCT
(scipy), orthogonality, closed forms for constant and basis blocks, exact
integer identities, a rigorous error bound, and interval proofs of the word
width.  A dropped term, a wrong sign, a swapped index or a wrong shift in
the flow graphs or the tables makes at least one of them fail.
"""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import codec, exact_dct, ijg, interval, linear, psnr, spec
from oracle.cordic_loeffler import Sigmas, cordic_gain, cordic_residual, gains

C8 = scipy.fft.dct(np.eye(8), type=2, norm="ortho", axis=0)


def test_spec_values():
    assert (spec.P, spec.N, spec.R, spec.QSHIFT, spec.DQ_CLAMP) == (4, 6, 11, 32, 4096)


def test_graph_converges_to_textbook_dct():
    # With many micro-rotations the CORDIC angles converge, and the graph
    # must become sqrt(8) * diag(g) * C exactly (pins every butterfly and
    # every rotation's inputs, outputs, angle and sign).
    a = linear.normalised_forward(40)
    assert np.abs(a - C8).max() < 1e-10


@pytest.mark.parametrize("n", [3, 4, 6, 8])
def test_graph_orthogonal_up_to_gain(n):
    a = linear.normalised_forward(n)
    assert np.abs(a @ a.T - np.eye(8)).max() < 1e-14


@pytest.mark.parametrize("n", [4, 6, 12])
def test_inverse_graph_is_transpose(n):
    assert np.abs(linear.inverse_matrix(n) - linear.forward_matrix(n).T).max() < 1e-14


def test_sigma_tables_and_residuals():
    s = Sigmas(6)
    assert s.odd_upper == (1, 1, -1, 1, -1, -1)
    assert s.odd_lower == (1, -1, -1, 1, 1, 1)
    assert s.even == (-1, 1, -1, -1, 1, -1)
    for ang, sig in ((3 * math.pi / 16, s.odd_upper), (math.pi / 16, s.odd_lower),
                     (-math.pi / 8, s.even)):
        # greedy CORDIC leaves at most the last micro-angle
        assert abs(cordic_residual(ang, sig)) <= math.atan(2.0 ** -6)


def test_gain_closed_form():
    k = cordic_gain(6)
    assert abs(k - math.prod(math.sqrt(1 + 4.0 ** -i) for i in range(1, 7))) < 1e-15
    assert abs(k - 1.1643879666) < 1e-9
    g = gains(6)
    assert g[0] == 1.0 and g[4] == 1.0 and g[1] == g[7] == k
    assert all(abs(g[i] - k / math.sqrt(2)) < 1e-15 for i in (2, 3, 5, 6))


@pytest.mark.parametrize("c", list(range(256)))
def test_constant_block_dc_only(c):
    # The DC path is adds only and every difference is 0: Y00 = 64 (c-128) 2^P, rest 0.
    y = codec.forward_coefficients(np.full((1, 8, 8), c, dtype=np.uint8))
    assert y[0, 0, 0] == 64 * (c - 128) * (1 << spec.P)
    y[0, 0, 0] = 0
    assert not y.any()


def test_constant_block_round_trip_exact():
    Q = ijg.luma_table(100)
    b = np.arange(256, dtype=np.uint8).reshape(256, 1, 1) * np.ones((1, 8, 8), dtype=np.uint8)
    r = codec.reconstruct_blocks(codec.compress_blocks(b, Q), Q)
    assert (r == b).all()


def test_quantiser_matches_ideal_rounding_off_ties():
    # constant block: X00 = 8 (c - 128); q00 must be round_half_away(X00 / Q00)
    # whenever X00 / Q00 is not within 1e-6 of a half-integer tie.
    for qv in (1, 2, 3, 7, 16, 48, 99, 255):
        qtab = np.full((8, 8), qv)
        for c in range(0, 256, 3):
            x00 = 8.0 * (c - 128)
            ratio = abs(x00) / qv
            if abs(ratio - math.floor(ratio) - 0.5) < 1e-6:
                continue
            q = codec.compress_blocks(np.full((1, 8, 8), c, dtype=np.uint8), qtab)
            assert q[0, 0, 0] == int(math.copysign(math.floor(ratio + 0.5), x00))


@pytest.mark.parametrize("u0,v0", [(0, 1), (2, 0), (3, 5), (7, 7), (1, 6)])
def test_basis_block_concentrates_energy(u0, v0):
    i = np.arange(8).reshape(-1, 1)
    j = np.arange(8).reshape(1, -1)
    x = 127.0 * np.cos(math.pi * u0 * (2 * i + 1) / 16) * np.cos(math.pi * v0 * (2 * j + 1) / 16)
    b = np.clip(np.round(x + 128), 0, 255).astype(np.uint8).reshape(1, 8, 8)
    y = codec.forward_coefficients(b)[0].astype(np.float64)
    xs = y / (8.0 * (1 << spec.P) * np.outer(gains(), gains()))
    e = xs * xs
    assert e[u0, v0] / e.sum() > 0.99


def test_error_bound_is_small_and_holds():
    bound = linear.cordic_vs_exact_bound()
    # stated bound at N = 6, P = 4 on the orthonormal scale (|X| <= 1024):
    # 13.85 worst case from the angle residuals (L1 over the block) plus the
    # truncation part (<= 1.3); random blocks stay near 4.4
    assert bound.max() < 14.0
    rng = np.random.default_rng(5)
    blocks = [rng.integers(0, 256, size=(4000, 8, 8)).astype(np.uint8)]
    # adversarial: sign patterns of the basis functions at full swing
    for u in range(8):
        for v in range(8):
            s = np.sign(np.outer(C8[u], C8[v]))
            s[s == 0] = 1
            blocks.append(np.where(s > 0, 255, 0).astype(np.uint8)[None])
            blocks.append(np.where(s > 0, 0, 255).astype(np.uint8)[None])
    b = np.concatenate(blocks)
    y = codec.forward_coefficients(b).astype(np.float64)
    xs = y / (8.0 * (1 << spec.P) * np.outer(gains(), gains()))
    xe = exact_dct.dct2(b.astype(np.float64) - 128.0)
    assert (np.abs(xs - xe) <= bound + 1e-9).all()


def test_fixed_point_round_trip_quality_100():
    rng = np.random.default_rng(6)
    b = rng.integers(0, 256, size=(5000, 8, 8)).astype(np.uint8)
    Q = ijg.luma_table(100)
    r = codec.reconstruct_blocks(codec.compress_blocks(b, Q), Q)
    assert np.abs(r.astype(int) - b.astype(int)).max() <= 2


def test_word_width_interval_proofs():
    f_row, f_col, _ = interval.forward_bounds()
    i_col, i_row = interval.inverse_bounds()
    assert max(f_row, f_col, i_col, i_row) < 2 ** 31
    # the GPU folds the descale rounding term and +128 into the DC input
    i_col2, i_row2 = interval.inverse_bounds(dc_offset=(1 << (spec.R + 2)) + (128 << (spec.R + 3)))
    assert max(i_col2, i_row2) < 2 ** 31
    bits, _ = interval.worst_case_product_bits(f_col)
    assert bits <= 63


def test_forward_output_fits_quantiser_contract():
    # |Y| < 2^31 and M < 2^32, so |Y| * M + 2^31 fits 64 unsigned bits, and
    # every quantised value fits int16.
    _, f_col, _ = interval.forward_bounds()
    m = codec.quant_multipliers(np.ones((8, 8)))
    assert m.max() < 2 ** 32 and m.min() > 0
    assert f_col * m.max() / 2.0 ** 32 + 1 < 2 ** 15


def test_tables_closed_form_entries():
    # (0,0): g = 1, so M00 = rint(2^25 / Q00) and W00 = 2^R exactly
    q = ijg.luma_table(50)
    m = codec.quant_multipliers(q)
    w = codec.dequant_weights()
    assert m[0, 0] == round(2 ** 25 / 16)
    assert w[0, 0] == 2 ** spec.R
    k = cordic_gain(6)
    assert w[1, 1] == int(np.rint(2 ** spec.R / (k * k)))
    assert w[2, 2] == int(np.rint(2 ** spec.R / (k * k / 2)))


def test_cordic_psnr_close_to_exact_table3_claim():
    # Tables 3-4: the Cordic-based transform's PSNR trails the exact DCT's.
    # At N = 6 the fixed-point transform is within a few hundredths of a dB.
    from synth import sinusoid_image
    img = sinusoid_image(128, 128, seed=0).numpy()
    for quality in (25, 50, 90):
        Q = ijg.luma_table(quality)
        c = codec.compress_plane(img, Q)
        r = codec.reconstruct_plane(c, Q, *img.shape)
        b = codec.plane_to_blocks(img).reshape(-1, 8, 8)
        re = exact_dct.exact_reconstruct_blocks(exact_dct.exact_compress_blocks(b, Q), Q)
        re = codec.blocks_to_plane(re.reshape(16, 16, 8, 8), *img.shape)
        p_c, p_e = psnr.psnr(img, r), psnr.psnr(img, re)
        assert p_c <= p_e + 0.05
        assert p_c >= p_e - 0.5


def test_padding_is_edge_replication():
    img = np.arange(13 * 7, dtype=np.uint8).reshape(13, 7)
    p = codec.pad_plane(img)
    assert p.shape == (16, 8)
    assert (p[:13, :7] == img).all()
    assert (p[13:, :7] == img[12]).all()
    assert (p[:13, 7] == img[:, 6]).all()
    blocks = codec.plane_to_blocks(img)
    assert blocks.shape == (2, 1, 8, 8)
    assert (codec.blocks_to_plane(blocks, 13, 7) == img).all()


def test_sigma_order_matters_for_truncated_inverse():
    # The transposed micro-rotations do not commute once truncated, so the
    # spec fixes ascending order; a descending-order inverse must differ on
    # some input (guards against silently reordering the inverse).
    from oracle.cordic_loeffler import cordic_rotate_t
    sig = Sigmas(6).odd_upper
    rng = np.random.default_rng(7)
    a = rng.integers(-100000, 100000, size=2000)
    b = rng.integers(-100000, 100000, size=2000)
    asc = cordic_rotate_t(a, b, sig)
    # descending order by hand
    x, y = a, b
    for i in range(6, 0, -1):
        s = sig[i - 1]
        x, y = (x - (y >> i), y + (x >> i)) if s > 0 else (x + (y >> i), y - (x >> i))
    assert (asc[0] != x).any() or (asc[1] != y).any()

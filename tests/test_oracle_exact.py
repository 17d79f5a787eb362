"""Pins for the FP64 textbook DCT (Eq. 3, 4, 6, 7) and the exact pipeline."""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import exact_dct, ijg, psnr


def test_matrix_is_scipy_orthonormal_dct2():
    # special case that reduces to a library routine: DCT-II, norm="ortho"
    ref = scipy.fft.dct(np.eye(8), type=2, norm="ortho", axis=0)
    assert np.allclose(exact_dct.dct_matrix(8), ref, atol=1e-15)


def test_dct2_matches_scipy_dctn():
    rng = np.random.default_rng(1)
    x = rng.uniform(-128, 127, size=(50, 8, 8))
    ref = scipy.fft.dctn(x, type=2, norm="ortho", axes=(-2, -1))
    assert np.allclose(exact_dct.dct2(x), ref, atol=1e-11)


def test_dct2_bruteforce_double_sum_tiny():
    rng = np.random.default_rng(2)
    f = rng.uniform(-128, 127, size=(8, 8))
    F = exact_dct.dct2(f)
    for u in (0, 1, 5, 7):
        for v in (0, 3, 6):
            s = 0.0
            for i in range(8):
                for j in range(8):
                    s += (math.cos(math.pi * u * (2 * i + 1) / 16) *
                          math.cos(math.pi * v * (2 * j + 1) / 16) * f[i, j])
            s *= 0.25 * exact_dct.alpha(u) * exact_dct.alpha(v)
            assert abs(s - F[u, v]) < 1e-10


@pytest.mark.parametrize("c", [0, 1, 64, 127, 128, 129, 200, 255])
def test_constant_block_only_dc(c):
    x = np.full((8, 8), c - 128.0)
    F = exact_dct.dct2(x)
    assert abs(F[0, 0] - 8.0 * (c - 128)) < 1e-12
    F[0, 0] = 0.0
    assert np.abs(F).max() < 1e-12


@pytest.mark.parametrize("u0,v0", [(0, 1), (1, 0), (3, 5), (7, 7), (4, 2)])
def test_cosine_basis_gives_one_coefficient(u0, v0):
    i = np.arange(8).reshape(-1, 1)
    j = np.arange(8).reshape(1, -1)
    x = np.cos(math.pi * u0 * (2 * i + 1) / 16) * np.cos(math.pi * v0 * (2 * j + 1) / 16)
    F = exact_dct.dct2(x)
    expect = 4.0 / (exact_dct.alpha(u0) * exact_dct.alpha(v0))   # 1 / (c_u c_v) with c = sqrt(2/8) alpha
    assert abs(F[u0, v0] - expect) < 1e-12
    F[u0, v0] = 0.0
    assert np.abs(F).max() < 1e-12


def test_parseval_and_round_trip():
    rng = np.random.default_rng(3)
    x = rng.uniform(-128, 127, size=(200, 8, 8))
    F = exact_dct.dct2(x)
    e_x = (x * x).sum(axis=(1, 2))
    e_f = (F * F).sum(axis=(1, 2))
    assert np.max(np.abs(e_x - e_f) / e_x) < 1e-12
    assert np.abs(exact_dct.idct2(F) - x).max() < 1e-11


def test_exact_pipeline_quality_100_is_near_lossless():
    rng = np.random.default_rng(4)
    b = rng.integers(0, 256, size=(300, 8, 8)).astype(np.uint8)
    Q = ijg.luma_table(100)
    assert (Q == 1).all()
    r = exact_dct.exact_reconstruct_blocks(exact_dct.exact_compress_blocks(b, Q), Q)
    # integer rounding of 64 coefficients by at most 1/2 each: |error| <= 4 (L2 -> Linf bound)
    assert np.abs(r.astype(int) - b.astype(int)).max() <= 4
    assert psnr.psnr(b, r) > 50.0


def test_exact_pipeline_quantiser_rounding():
    # X00 = 8 (c - 128); with Q00 = 16 at quality 50, q00 = round_half_away(X00 / 16)
    Q = ijg.luma_table(50)
    for c in range(256):
        b = np.full((1, 8, 8), c, dtype=np.uint8)
        q = exact_dct.exact_compress_blocks(b, Q)
        x00 = 8.0 * (c - 128)
        ratio = abs(x00) / 16.0
        if abs(ratio - math.floor(ratio) - 0.5) > 1e-6:     # FP64 noise decides exact ties
            assert q[0, 0, 0] == int(math.copysign(math.floor(ratio + 0.5), x00))
        assert np.abs(q[0]).sum() == abs(q[0, 0, 0])


def test_fp32_pipeline_matches_fp64_definition():
    """The float32 exact pipeline (fixed operation order, as the GPU runs
    it) against the FP64 definition of Eq. 6: identical codes except where
    |X|/Q sits within float32 rounding of a .5 tie, reconstructions within 1,
    PSNR within 0.01 dB."""
    from oracle import exact_fp32
    rng = np.random.default_rng(12)
    b = rng.integers(0, 256, size=(3000, 8, 8)).astype(np.uint8)
    for quality in (10, 50, 90, 100):
        Q = ijg.luma_table(quality)
        q64 = exact_dct.exact_compress_blocks(b, Q)
        q32 = exact_fp32.compress_blocks(b, Q).astype(np.int64)
        X = exact_dct.dct2(b.astype(np.float64) - 128.0)
        frac = np.abs(X) / Q - np.floor(np.abs(X) / Q)
        near_tie = np.abs(frac - 0.5) < 1e-4
        assert np.array_equal(q32[~near_tie], q64[~near_tie])
        assert np.abs(q32 - q64).max() <= 1
        r64 = exact_dct.exact_reconstruct_blocks(q64, Q)
        r32 = exact_fp32.reconstruct_blocks(q64, Q)
        assert np.abs(r32.astype(int) - r64.astype(int)).max() <= 1
        assert abs(psnr.psnr(b, r32) - psnr.psnr(b, r64)) < 0.01


def test_fp32_pipeline_constant_blocks():
    from oracle import exact_fp32
    b = np.arange(256, dtype=np.uint8).reshape(256, 1, 1) * np.ones((1, 8, 8), dtype=np.uint8)
    Q = ijg.luma_table(100)
    r = exact_fp32.reconstruct_blocks(exact_fp32.compress_blocks(b, Q), Q)
    assert np.abs(r.astype(int) - b.astype(int)).max() <= 1

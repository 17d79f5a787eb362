"""Pins for SSE/PSNR (Eq. 23, 24) and the IJG quality scaling."""
import math

import numpy as np
import pytest

from oracle import ijg, psnr


def test_psnr_off_by_one_closed_form():
    o = np.full((20, 30), 100, dtype=np.uint8)
    c = o + 1
    assert psnr.sse(o, c) == 600
    assert abs(psnr.psnr(o, c) - 20.0 * math.log10(255.0)) < 1e-12
    assert abs(psnr.psnr(o, c) - 48.13080360867910) < 1e-9


def test_psnr_identical_is_infinite():
    o = np.arange(64, dtype=np.uint8).reshape(8, 8)
    assert psnr.psnr(o, o) == math.inf


def test_psnr_matches_eq23_literal():
    rng = np.random.default_rng(8)
    o = rng.integers(0, 256, size=(37, 41)).astype(np.uint8)
    c = np.clip(o.astype(int) + rng.integers(-9, 10, size=o.shape), 0, 255).astype(np.uint8)
    assert abs(psnr.psnr(o, c) - psnr.psnr_eq23(o, c)) < 1e-9
    mx = float(o.max())
    assert abs(psnr.psnr(o, c, max_of_original=True) - psnr.psnr_eq23(o, c, mx)) < 1e-9


def test_sse_bruteforce_loops():
    rng = np.random.default_rng(9)
    o = rng.integers(0, 256, size=(5, 7)).astype(np.uint8)
    c = rng.integers(0, 256, size=(5, 7)).astype(np.uint8)
    s = 0
    for i in range(5):
        for j in range(7):
            s += (int(o[i, j]) - int(c[i, j])) ** 2
    assert psnr.sse(o, c) == s


def test_ijg_closed_forms():
    assert (ijg.luma_table(50) == ijg.LUMA_BASE).all()
    assert (ijg.chroma_table(50) == ijg.CHROMA_BASE).all()
    assert (ijg.luma_table(100) == 1).all()
    assert (ijg.luma_table(1) == 255).all()
    assert int(ijg.LUMA_BASE.sum()) == 3688
    assert int(ijg.CHROMA_BASE.sum()) == 17 + 18 + 24 + 47 + 18 + 21 + 26 + 66 + 24 + 26 + 56 + 47 + 66 + 99 * 51
    # quality 75: s = 50, Q = (16 * 50 + 50) // 100 = 8 at (0, 0)
    assert ijg.luma_table(75)[0, 0] == 8
    # quality 10: s = 500, Q = (16 * 500 + 50) // 100 = 80
    assert ijg.luma_table(10)[0, 0] == 80


@pytest.mark.parametrize("q", [0, 101, -5])
def test_ijg_rejects_out_of_range(q):
    with pytest.raises(ValueError):
        ijg.luma_table(q)


def test_ijg_monotone_in_quality():
    prev = None
    for q in range(1, 101):
        t = ijg.luma_table(q)
        if prev is not None:
            assert (t <= prev).all()
        prev = t

"""Pins for the RGB -> YCbCr 4:2:0 oracle: coefficient derivation, grey
invariance, JFIF reference colours, a float64 reference and the 2x2 mean."""
import numpy as np

from oracle import color


def test_coefficients_are_rounded_jfif_values():
    k = {"y": (0.299, 0.587, 0.114), "cb": (-0.168736, -0.331264, 0.5), "cr": (0.5, -0.418688, -0.081312)}
    assert color.Y_COEF == tuple(int(round(v * 65536)) for v in k["y"])
    assert color.CB_COEF == tuple(int(round(v * 65536)) for v in k["cb"])
    assert color.CR_COEF == tuple(int(round(v * 65536)) for v in k["cr"])
    assert sum(color.Y_COEF) == 65536 and sum(color.CB_COEF) == 0 and sum(color.CR_COEF) == 0


def test_grey_maps_to_neutral_chroma():
    v = np.arange(256, dtype=np.uint8)
    rgb = np.stack([v, v, v], axis=-1)[None]
    y, cb, cr = color.full_res(rgb)
    assert (y[0] == v).all() and (cb == 128).all() and (cr == 128).all()


def test_primary_colours():
    rgb = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255], [0, 0, 0]]], dtype=np.uint8)
    y, cb, cr = color.full_res(rgb)
    assert y[0].tolist() == [76, 150, 29, 255, 0]
    assert cb[0].tolist() == [85, 44, 255, 128, 128]
    assert cr[0].tolist() == [255, 21, 107, 128, 128]


def test_matches_float_reference_within_one():
    rng = np.random.default_rng(1)
    rgb = rng.integers(0, 256, size=(40, 52, 3)).astype(np.float64)
    r, g, b = rgb[..., 0], rgb[..., 1], rgb[..., 2]
    yf = 0.299 * r + 0.587 * g + 0.114 * b
    cbf = np.clip(-0.168736 * r - 0.331264 * g + 0.5 * b + 128, 0, 255)
    crf = np.clip(0.5 * r - 0.418688 * g - 0.081312 * b + 128, 0, 255)
    y, cb, cr = color.full_res(rgb.astype(np.uint8))
    assert np.abs(y - yf).max() <= 0.51 and np.abs(cb - cbf).max() <= 0.51 and np.abs(cr - crf).max() <= 0.51


def test_subsample_is_rounded_mean_with_edge_repeat():
    c = np.arange(5 * 7, dtype=np.int64).reshape(5, 7)
    s = color.subsample(c)
    assert s.shape == (3, 4)
    assert s[0, 0] == (c[0, 0] + c[0, 1] + c[1, 0] + c[1, 1] + 2) >> 2
    assert s[2, 3] == c[4, 6]                       # corner: one pixel repeated four times
    assert s[1, 3] == (2 * c[2, 6] + 2 * c[3, 6] + 2) >> 2

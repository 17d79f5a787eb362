"""RGB to YCbCr 4:2:0 conversion (no counterpart in the paper, which works on
grey images; colour input for the 4:2:0 workloads).

Full-range BT.601 as in JFIF, in integer arithmetic with 16-bit fixed-point
coefficients c = rint(k * 65536) of
  Y  =  0.299 R + 0.587 G + 0.114 B
  Cb = -0.168736 R - 0.331264 G + 0.5 B + 128
  Cr =  0.5 R - 0.418688 G - 0.081312 B + 128
(each row's integer coefficients sum to 65536, 0, 0):
  Y  = (19595 R + 38470 G + 7471 B + 32768) >> 16
  Cb = clamp((-11058 R - 21710 G + 32768 B + (128 << 16) + 32768) >> 16, 0, 255)
  Cr = clamp((32768 R - 27439 G - 5329 B + (128 << 16) + 32768) >> 16, 0, 255)
Chroma is computed per pixel, then averaged over 2x2 with rounding,
(a + b + c + d + 2) >> 2; an odd last row or column repeats its edge pixel.

Test infrastructure only (see the package docstring).
"""
import numpy as np

Y_COEF = (19595, 38470, 7471)
CB_COEF = (-11058, -21710, 32768)
CR_COEF = (32768, -27439, -5329)


def full_res(rgb):
    """rgb: (H, W, 3) uint8 -> (Y, Cb, Cr) full-resolution int64 planes."""
    r, g, b = (np.asarray(rgb, dtype=np.int64)[..., k] for k in range(3))
    y = (Y_COEF[0] * r + Y_COEF[1] * g + Y_COEF[2] * b + 32768) >> 16
    cb = np.clip((CB_COEF[0] * r + CB_COEF[1] * g + CB_COEF[2] * b + (128 << 16) + 32768) >> 16, 0, 255)
    cr = np.clip((CR_COEF[0] * r + CR_COEF[1] * g + CR_COEF[2] * b + (128 << 16) + 32768) >> 16, 0, 255)
    return y, cb, cr


def subsample(c):
    """2x2 average with rounding; odd sizes repeat the last row / column."""
    h, w = c.shape
    p = np.pad(c, ((0, h % 2), (0, w % 2)), mode="edge")
    s = p[0::2, 0::2] + p[0::2, 1::2] + p[1::2, 0::2] + p[1::2, 1::2]
    return (s + 2) >> 2


def rgb_to_yuv420(rgb):
    y, cb, cr = full_res(rgb)
    return y.astype(np.uint8), subsample(cb).astype(np.uint8), subsample(cr).astype(np.uint8)

"""Plane-level fixed-point codec: padding, level shift, 2-D Cordic-Loeffler
transform, quantiser, dequantiser, inverse transform, descale.

Sec. 3.2 runs the DCT, the quantiser and the IDCT as three separate steps;
this module keeps them as separate functions in that order.  The 2-D
transform is Eq. 6's separable form: the 8-point graph on every row, then
on every column; the inverse applies the transposed graph to the columns,
then to the rows (the exact transpose of the forward order).

Numeric reading (spec file): input x = (p - 128) * 2^P; the forward output
is Y_uv ~ 8 * 2^P * g_u * g_v * X_uv where X is the orthonormal 2-D DCT;
the quantiser multiplies by M_uv = rint(2^32 / (8 * 2^P * g_u g_v Q_uv)) and
rounds half away from zero; the dequantiser forms G = clamp(q Q, -4096,
4096) * W_uv with W_uv = rint(2^R / (g_u g_v)); two inverse passes give
~ 8 * 2^R * x, descaled by a rounding shift of R + 3 and shifted back by 128.
All intermediate values are checked to fit in int32.

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np

from . import spec
from .cordic_loeffler import Sigmas, gains, loeffler8_forward, loeffler8_inverse

INT32_LIMIT = 1 << 31


def _check_int32(a, what):
    m = int(np.abs(a).max()) if np.asarray(a).size else 0
    if m >= INT32_LIMIT:
        raise OverflowError("%s exceeds the int32 range (%d)" % (what, m))


def _along(fn, arr, axis, sig):
    """Apply an 8-point flow graph along ``axis`` of an integer array."""
    pts = [np.take(arr, k, axis=axis) for k in range(8)]
    return np.stack(fn(pts, sig), axis=axis)


# --------------------------------------------------------------------------
# tables
# --------------------------------------------------------------------------

def quant_multipliers(qtab, n=None, p=None):
    """M_uv = rint_half_even(2^(32-3-P) / ((g_u * g_v) * Q_uv)), int64.
    (2^32 / (8 * 2^P * g_u g_v Q) with the power of two taken out exactly.)"""
    n = spec.N if n is None else n
    p = spec.P if p is None else p
    g = gains(n)
    q = np.asarray(qtab, dtype=np.int64).reshape(8, 8)
    m = np.empty((8, 8), dtype=np.int64)
    for u in range(8):
        for v in range(8):
            den = (g[u] * g[v]) * float(q[u, v])
            m[u, v] = int(np.rint(math.ldexp(1.0, spec.QSHIFT - 3 - p) / den))
    return m


def dequant_weights(n=None, r=None):
    """W_uv = rint_half_even(2^R / (g_u * g_v)), int64."""
    n = spec.N if n is None else n
    r = spec.R if r is None else r
    g = gains(n)
    w = np.empty((8, 8), dtype=np.int64)
    for u in range(8):
        for v in range(8):
            w[u, v] = int(np.rint(math.ldexp(1.0, r) / (g[u] * g[v])))
    return w


# --------------------------------------------------------------------------
# block steps
# --------------------------------------------------------------------------

def level_shift(blocks_u8, p=None):
    """x = (p - 128) * 2^P as int64."""
    p = spec.P if p is None else p
    return (np.asarray(blocks_u8, dtype=np.int64) - 128) * (1 << p)


def forward_2d(x, sig=None):
    """Row pass then column pass of the forward graph on (..., 8, 8)."""
    sig = Sigmas() if sig is None else sig
    z = _along(loeffler8_forward, x, -1, sig)       # rows: points along j
    _check_int32(z, "forward row pass")
    y = _along(loeffler8_forward, z, -2, sig)       # columns: points along i
    _check_int32(y, "forward column pass")
    return y


def inverse_2d(g, sig=None):
    """Column pass then row pass of the transposed graph on (..., 8, 8)."""
    sig = Sigmas() if sig is None else sig
    t = _along(loeffler8_inverse, g, -2, sig)
    _check_int32(t, "inverse column pass")
    v = _along(loeffler8_inverse, t, -1, sig)
    _check_int32(v, "inverse row pass")
    return v


def quantize(y, m):
    """q = sgn(Y) * ((|Y| * M + 2^31) >> 32): rounding half away from zero."""
    a = np.abs(np.asarray(y, dtype=np.int64))
    q = (a * np.asarray(m, dtype=np.int64) + (1 << (spec.QSHIFT - 1))) >> spec.QSHIFT
    return np.where(np.asarray(y) < 0, -q, q)


def dequantize(q, qtab, w):
    """G = clamp(q * Q, -4096, 4096) * W."""
    t = np.asarray(q, dtype=np.int64) * np.asarray(qtab, dtype=np.int64)
    t = np.clip(t, -spec.DQ_CLAMP, spec.DQ_CLAMP)
    return t * np.asarray(w, dtype=np.int64)


def descale(v, r=None):
    """r = clamp(((v + 2^(R+2)) >> (R+3)) + 128, 0, 255) as uint8."""
    r = spec.R if r is None else r
    out = ((np.asarray(v, dtype=np.int64) + (1 << (r + 2))) >> (r + 3)) + 128
    return np.clip(out, 0, 255).astype(np.uint8)


def compress_blocks(blocks_u8, qtab, n=None):
    """(n, 8, 8) uint8 blocks -> (n, 8, 8) int16 quantised coefficients, with
    N = n CORDIC micro-rotations per rotation (None: the spec's)."""
    y = forward_2d(level_shift(blocks_u8), Sigmas(n))
    q = quantize(y, quant_multipliers(qtab, n))
    assert np.abs(q).max(initial=0) < (1 << 15)
    return q.astype(np.int16)


def reconstruct_blocks(coeffs, qtab, n=None):
    """(n, 8, 8) int16 coefficients -> (n, 8, 8) uint8 reconstructed blocks."""
    g = dequantize(coeffs, qtab, dequant_weights(n))
    return descale(inverse_2d(g, Sigmas(n)))


def forward_coefficients(blocks_u8, n=None):
    """The unquantised forward output Y (int64), for statistics."""
    return forward_2d(level_shift(blocks_u8), Sigmas(n))


# --------------------------------------------------------------------------
# planes
# --------------------------------------------------------------------------

def block_grid(height, width):
    """Number of block rows and block columns of an H x W plane."""
    return (height + 7) // 8, (width + 7) // 8


def pad_plane(img):
    """Edge replication up to multiples of 8 in both dimensions."""
    img = np.asarray(img, dtype=np.uint8)
    h, w = img.shape
    nby, nbx = block_grid(h, w)
    return np.pad(img, ((0, nby * 8 - h), (0, nbx * 8 - w)), mode="edge")


def plane_to_blocks(img):
    """(H, W) uint8 -> (nby, nbx, 8, 8) blocks of the edge-padded plane."""
    p = pad_plane(img)
    nby, nbx = p.shape[0] // 8, p.shape[1] // 8
    return p.reshape(nby, 8, nbx, 8).transpose(0, 2, 1, 3)


def blocks_to_plane(blocks, height, width):
    """(nby, nbx, 8, 8) -> (H, W): the padded area is dropped."""
    nby, nbx = blocks.shape[:2]
    full = blocks.transpose(0, 2, 1, 3).reshape(nby * 8, nbx * 8)
    return full[:height, :width]


def compress_plane(img, qtab, n=None):
    """uint8 (H, W) plane -> int16 coefficients (nby, nbx, 8, 8), block-major."""
    return compress_blocks(plane_to_blocks(img), qtab, n)


def reconstruct_plane(coeffs, qtab, height, width, n=None):
    """int16 (nby, nbx, 8, 8) coefficients -> uint8 (H, W) reconstruction."""
    return blocks_to_plane(reconstruct_blocks(coeffs, qtab, n), height, width)

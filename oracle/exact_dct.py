"""FP64 textbook DCT-II and its inverse, and the exact-DCT compression
pipeline used as the "DCT" row of Tables 3 and 4.

Eq. 3 defines the N-point 1-D DCT with the normalisation sqrt(2/N) and
alpha = 1/sqrt(2) at frequency 0 (Eq. 4); the printed formula attaches
alpha and the output to the wrong index (F(x), alpha(i)), which is read as
F(u) with alpha(u).  Eq. 6 is the separable 2-D form (its first cosine is
missing in print and alpha(i) alpha(j) is read as alpha(u) alpha(v)); Eq. 7
repeats the normalisation.

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np


def alpha(k):
    """Eq. 4 / Eq. 7: 1/sqrt(2) at frequency 0, else 1."""
    return 1.0 / math.sqrt(2.0) if k == 0 else 1.0


def dct_matrix(n):
    """Row u of the matrix is the u-th basis of Eq. 3:
    C[u, i] = sqrt(2/n) * alpha(u) * cos(pi * u * (2i + 1) / (2n))."""
    c = np.empty((n, n), dtype=np.float64)
    for u in range(n):
        for i in range(n):
            c[u, i] = math.sqrt(2.0 / n) * alpha(u) * math.cos(math.pi * u * (2 * i + 1) / (2.0 * n))
    return c


_C8 = dct_matrix(8)


def dct1(f):
    """Eq. 3 along the last axis (8 points)."""
    return np.asarray(f, dtype=np.float64) @ _C8.T


def idct1(F):
    """Inverse of Eq. 3: the transpose of the orthonormal matrix."""
    return np.asarray(F, dtype=np.float64) @ _C8


def dct2(block):
    """Eq. 6 on the last two axes of an (..., 8, 8) array:
    F(u, v) = sum_i sum_j C[u, i] C[v, j] f(i, j), i.e. C f C^T."""
    b = np.asarray(block, dtype=np.float64)
    return _C8 @ b @ _C8.T


def idct2(coef):
    """Inverse of Eq. 6: C^T F C."""
    c = np.asarray(coef, dtype=np.float64)
    return _C8.T @ c @ _C8


def exact_compress_blocks(blocks_u8, qtab):
    """Exact pipeline, quantiser step: X = DCT2(p - 128),
    q = sgn(X) * floor(|X| / Q + 1/2) (JPEG rounding, half away from zero).
    blocks_u8: (n, 8, 8) uint8; qtab: (8, 8) integers.  Returns int64 q."""
    x = np.asarray(blocks_u8, dtype=np.float64) - 128.0
    X = dct2(x)
    Q = np.asarray(qtab, dtype=np.float64)
    return (np.sign(X) * np.floor(np.abs(X) / Q + 0.5)).astype(np.int64)


def exact_reconstruct_blocks(q, qtab):
    """Exact pipeline, dequantiser + IDCT: x = IDCT2(q * Q) + 128,
    r = clamp(floor(x + 1/2), 0, 255)."""
    X = np.asarray(q, dtype=np.float64) * np.asarray(qtab, dtype=np.float64)
    x = idct2(X) + 128.0
    return np.clip(np.floor(x + 0.5), 0, 255).astype(np.uint8)

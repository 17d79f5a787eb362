"""The exact-DCT compression pipeline (the "DCT" rows of Tables 3 and 4) in
float32 with a fixed order of operations, as the GPU computes it.

Floating point decides integer results here (the quantised codes, the
rounded pixels), so both sides take those decisions in the same precision
and order.  Definition (all arithmetic float32, each product and each sum
rounded on its own, no fused multiply-add):

  C32[u][i]  = float32 of the FP64 value sqrt(2/8) alpha(u) cos(pi u (2i+1) / 16)
  rows       Z[i][v] = ((C32[v][0] x[i][0] + C32[v][1] x[i][1]) + ...) + C32[v][7] x[i][7]
  columns    X[u][v] = ((C32[u][0] Z[0][v] + C32[u][1] Z[1][v]) + ...) + C32[u][7] Z[7][v]
  quantise   q = sgn(X) floor(|X| / Q + 0.5)            (x = p - 128)
  dequantise D = q Q
  columns    T[i][v] = sum over u ascending of C32[u][i] D[u][v]
  rows       y[i][j] = sum over v ascending of C32[v][j] T[i][v]
  pixel      r = clamp(floor((y + 128) + 0.5), 0, 255)

It is Eq. 6 (and its inverse) evaluated in single precision; the tests pin it
to the FP64 pipeline of ``exact_dct``.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from .exact_dct import dct_matrix

C32 = dct_matrix(8).astype(np.float32)
F32 = np.float32


def _matvec_rows(c, x):
    """out[..., i, v] = sum_k c[v, k] * x[..., i, k], k ascending, float32."""
    out = np.empty_like(x)
    for v in range(8):
        acc = c[v, 0] * x[..., :, 0]
        for k in range(1, 8):
            acc = acc + c[v, k] * x[..., :, k]
        out[..., :, v] = acc
    return out


def _matvec_cols(c, z):
    """out[..., u, v] = sum_k c[u, k] * z[..., k, v], k ascending, float32."""
    out = np.empty_like(z)
    for u in range(8):
        acc = c[u, 0] * z[..., 0, :]
        for k in range(1, 8):
            acc = acc + c[u, k] * z[..., k, :]
        out[..., u, :] = acc
    return out


def forward(blocks_u8):
    x = np.asarray(blocks_u8, dtype=np.float32) - F32(128.0)
    return _matvec_cols(C32, _matvec_rows(C32, x))


def quantize(X, qtab):
    Q = np.asarray(qtab, dtype=np.float32).reshape(8, 8)
    t = np.floor(np.abs(X) / Q + F32(0.5))
    return (np.sign(X) * t).astype(np.int64)


def compress_blocks(blocks_u8, qtab):
    q = quantize(forward(blocks_u8), qtab)
    assert np.abs(q).max(initial=0) < (1 << 15)
    return q.astype(np.int16)


def reconstruct_blocks(q, qtab):
    D = np.asarray(q, dtype=np.float32) * np.asarray(qtab, dtype=np.float32).reshape(8, 8)
    ct = np.ascontiguousarray(C32.T)          # inverse: transposed basis
    T = _matvec_cols(ct, D)
    y = _matvec_rows(ct, T)
    r = np.floor((y + F32(128.0)) + F32(0.5))
    return np.clip(r, 0, 255).astype(np.uint8)

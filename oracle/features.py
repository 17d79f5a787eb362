"""Per-image statistics and the 80 inputs of the learned rate controller.

The paper has no rate controller; the statistics are those the forward pass
(Sec. 2.5.2 transform) can gather in integer arithmetic while it runs, and
the 80 features are fixed functions of them:

statistics words of a plane (over all 8x8 blocks of the edge-padded plane):
  [0..63]  band energy E_uv = sum over blocks of (|Y_uv| >> (P + 1))^2,
           Y the unquantised fixed-point forward output
  [64] sum p   [65] sum p^2   [66] min p   [67] max p
  [68] sum |dx|   [69] sum |dy|   [70] sum dx^2   [71] sum dy^2
           (dx, dy: differences of neighbouring samples inside a block)
  [72..75] number of blocks whose AC energy sum_{(u,v) != (0,0)} of
           (|Y_uv| >> (P + 1))^2 is below 2^10, 2^14, 2^18, 2^22
  [76] blocks   [77] samples (64 per block)   [78, 79] zero

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np

from . import spec
from .codec import forward_coefficients, plane_to_blocks

STATS_WORDS = 80
N_FEATURES = 80


def block_stats(blocks_u8):
    """Statistics words (80 Python ints) of an (n, 8, 8) uint8 block set."""
    b = np.asarray(blocks_u8, dtype=np.int64).reshape(-1, 8, 8)
    y = forward_coefficients(b.astype(np.uint8))
    a = np.abs(y) >> (spec.P + 1)
    e = a * a
    out = [0] * STATS_WORDS
    band = e.sum(axis=0)
    for u in range(8):
        for v in range(8):
            out[u * 8 + v] = int(band[u, v])
    out[64] = int(b.sum())
    out[65] = int((b * b).sum())
    out[66] = int(b.min()) if b.size else 255
    out[67] = int(b.max()) if b.size else 0
    dx = b[:, :, 1:] - b[:, :, :-1]
    dy = b[:, 1:, :] - b[:, :-1, :]
    out[68] = int(np.abs(dx).sum())
    out[69] = int(np.abs(dy).sum())
    out[70] = int((dx * dx).sum())
    out[71] = int((dy * dy).sum())
    ac = e.reshape(-1, 64)[:, 1:].sum(axis=1)
    for k in range(4):
        out[72 + k] = int((ac < (1 << (10 + 4 * k))).sum())
    out[76] = int(b.shape[0])
    out[77] = int(b.shape[0] * 64)
    return out


def plane_stats(img):
    """Statistics words of a uint8 (H, W) plane (edge-padded to blocks)."""
    return block_stats(plane_to_blocks(img).reshape(-1, 8, 8))


def features_from_stats(st, width, height, target_psnr):
    """The 80 controller inputs (float64) from the statistics words:
      0..63  log(1 + E_uv / blocks)  (mean squared band amplitude, log scale)
      64 mean/128, 65 std/64, 66 min/255, 67 max/255,
      68 mean|dx|/32, 69 mean|dy|/32, 70 sqrt(mean dx^2)/32, 71 sqrt(mean dy^2)/32,
      72..75 fraction of blocks below each AC energy threshold,
      76 log2(W)/11, 77 log2(H)/11, 78 (target - 35)/7, 79 1 (bias)."""
    nb = float(st[76])
    ns = float(st[77])
    f = np.zeros(N_FEATURES, dtype=np.float64)
    for k in range(64):
        f[k] = math.log1p(st[k] / nb)
    mean = st[64] / ns
    var = max(st[65] / ns - mean * mean, 0.0)
    f[64] = mean / 128.0
    f[65] = math.sqrt(var) / 64.0
    f[66] = st[66] / 255.0
    f[67] = st[67] / 255.0
    nd = nb * 56.0
    f[68] = st[68] / nd / 32.0
    f[69] = st[69] / nd / 32.0
    f[70] = math.sqrt(st[70] / nd) / 32.0
    f[71] = math.sqrt(st[71] / nd) / 32.0
    for k in range(4):
        f[72 + k] = st[72 + k] / nb
    f[76] = math.log2(width) / 11.0
    f[77] = math.log2(height) / 11.0
    f[78] = (target_psnr - 35.0) / 7.0
    f[79] = 1.0
    return f

"""JPEG base quantisation tables and the IJG quality scaling.

The paper runs a separate quantiser kernel (Sec. 3.2) but prints no table or
quality; the workloads use the ITU-T T.81 Annex K example tables scaled by
the Independent JPEG Group's quality rule.  Tables are in natural (row u,
column v) order, not zig-zag.

Test infrastructure only (see the package docstring).
"""
import numpy as np

# ITU-T T.81 Annex K, Table K.1 (luminance), natural order.
LUMA_BASE = np.array([
    [16, 11, 10, 16, 24, 40, 51, 61],
    [12, 12, 14, 19, 26, 58, 60, 55],
    [14, 13, 16, 24, 40, 57, 69, 56],
    [14, 17, 22, 29, 51, 87, 80, 62],
    [18, 22, 37, 56, 68, 109, 103, 77],
    [24, 35, 55, 64, 81, 104, 113, 92],
    [49, 64, 78, 87, 103, 121, 120, 101],
    [72, 92, 95, 98, 112, 100, 103, 99],
], dtype=np.int64)

# ITU-T T.81 Annex K, Table K.2 (chrominance), natural order.
CHROMA_BASE = np.full((8, 8), 99, dtype=np.int64)
CHROMA_BASE[0, :4] = [17, 18, 24, 47]
CHROMA_BASE[1, :4] = [18, 21, 26, 66]
CHROMA_BASE[2, :3] = [24, 26, 56]
CHROMA_BASE[3, :2] = [47, 66]


def quality_scale(quality):
    """IJG percentage scale: 5000/q below 50, 200 - 2q from 50 up (integers)."""
    q = int(quality)
    if q < 1 or q > 100:
        raise ValueError("quality must be in 1..100")
    return 5000 // q if q < 50 else 200 - 2 * q


def scaled_table(base, quality):
    """Q = clamp((base * s + 50) / 100, 1, 255) with integer division."""
    s = quality_scale(quality)
    t = (np.asarray(base, dtype=np.int64) * s + 50) // 100
    return np.clip(t, 1, 255).astype(np.int64)


def luma_table(quality):
    return scaled_table(LUMA_BASE, quality)


def chroma_table(quality):
    return scaled_table(CHROMA_BASE, quality)

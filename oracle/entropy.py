"""Rate of the quantised coefficients (no counterpart in the paper, which
never measures the compressed size): the JPEG-style symbol stream of each
plane and its ideal static entropy code length.

Per block, in block-major order:
  DC   d = q00 - q00(previous block of the plane) (0 for the first block);
       symbol = category(d) in 0..15, plus category(d) amplitude bits
  AC   the 63 coefficients in zig-zag order; a run of 16 zeros before a
       non-zero value emits ZRL = 0xF0; a non-zero value v after r < 16 zeros
       emits (r << 4) | category(v) plus category(v) amplitude bits; trailing
       zeros emit EOB = 0x00
category(v) = number of bits of |v| (0 for v = 0).  With the symbol counts
n_s (DC and AC separately, N = sum n_s) the plane costs
  bits = amplitude bits + sum_s n_s log2(N / n_s)
which is what an ideal static code for that plane's own statistics spends.

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np


def zigzag():
    """Natural index u*8+v of the k-th zig-zag position: diagonals s = u+v in
    turn, odd s with u rising, even s with u falling."""
    order = []
    for s in range(15):
        us = range(max(0, s - 7), min(s, 7) + 1)
        us = us if s % 2 else reversed(us)
        order.extend(u * 8 + (s - u) for u in us)
    return order


ZIGZAG = zigzag()


def category(v):
    return int(abs(int(v))).bit_length()


def plane_histograms(coeffs):
    """coeffs: (nblk, 64) integers in natural order, block-major.  Returns
    (dc_hist[16], ac_hist[256], amplitude bits, blocks) as Python ints."""
    c = np.asarray(coeffs, dtype=np.int64).reshape(-1, 64)
    dc = np.zeros(16, dtype=np.int64)
    ac = np.zeros(256, dtype=np.int64)
    amp = 0
    prev = 0
    for blk in c:
        d = int(blk[0]) - prev
        prev = int(blk[0])
        k = category(d)
        dc[k] += 1
        amp += k
        run = 0
        for z in ZIGZAG[1:]:
            v = int(blk[z])
            if v == 0:
                run += 1
                continue
            while run >= 16:
                ac[0xF0] += 1
                run -= 16
            s = category(v)
            ac[(run << 4) | s] += 1
            amp += s
            run = 0
        if run:
            ac[0x00] += 1
    return [int(v) for v in dc], [int(v) for v in ac], amp, c.shape[0]


def entropy_bits(hist):
    n = sum(hist)
    return sum(h * math.log2(n / h) for h in hist if h)


def plane_bits(coeffs):
    dc, ac, amp, _ = plane_histograms(coeffs)
    return amp + entropy_bits(dc) + entropy_bits(ac)

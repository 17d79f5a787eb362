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
An achievable count: the plane's DC symbols and its AC symbols each get an
optimal prefix code whose codewords are at most 16 bits long (the limit of
JPEG's Huffman tables), found by the package-merge method of Larmore and
Hirschberg; the plane then costs
  bits = amplitude bits + sum_s n_s len_s(DC) + sum_s n_s len_s(AC)
with a lone symbol coded in one bit.

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


def limited_code_lengths(counts, max_len=16):
    """Codeword lengths of an optimal prefix code over the symbols with
    non-zero counts, no codeword longer than max_len (package-merge).
    Returns a list aligned with ``counts`` (0 for absent symbols)."""
    live = [i for i, c in enumerate(counts) if c > 0]
    lengths = [0] * len(counts)
    if not live:
        return lengths
    if len(live) == 1:
        lengths[live[0]] = 1
        return lengths
    if len(live) > (1 << max_len):
        raise ValueError("too many symbols for the length limit")
    # An item is (weight, per-leaf multiplicity).  The leaves, sorted by
    # weight (ties by symbol index), seed every level; level by level the
    # sorted list is packaged in adjacent pairs and merged with the leaves.
    leaves = sorted(((counts[i], i) for i in live))
    leaf_items = [(w, {i: 1}) for w, i in leaves]

    def merge(a, b):
        out, x, y = [], 0, 0
        while x < len(a) or y < len(b):
            if y == len(b) or (x < len(a) and a[x][0] <= b[y][0]):
                out.append(a[x])
                x += 1
            else:
                out.append(b[y])
                y += 1
        return out

    current = list(leaf_items)
    for _ in range(max_len - 1):
        packages = []
        for k in range(0, len(current) - 1, 2):
            wa, ma = current[k]
            wb, mb = current[k + 1]
            m = dict(ma)
            for key, v in mb.items():
                m[key] = m.get(key, 0) + v
            packages.append((wa + wb, m))
        current = merge(leaf_items, packages)
    for _, m in current[:2 * len(live) - 2]:
        for key, v in m.items():
            lengths[key] += v
    return lengths


def code_cost(counts, max_len=16):
    """Bits of the symbols under limited_code_lengths."""
    return sum(c * l for c, l in zip(counts, limited_code_lengths(counts, max_len)))


def plane_huffman_bits(coeffs):
    dc, ac, amp, _ = plane_histograms(coeffs)
    return amp + code_cost(dc) + code_cost(ac)

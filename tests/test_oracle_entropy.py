"""Pins for the rate oracle: the zig-zag order, symbol counts on hand-made
blocks, and the entropy code length."""
import math

import numpy as np

from oracle import entropy

# ITU-T T.81 Figure A.6 zig-zag sequence, natural indices
ZZ = [0, 1, 8, 16, 9, 2, 3, 10, 17, 24, 32, 25, 18, 11, 4, 5, 12, 19, 26, 33, 40, 48, 41, 34, 27, 20, 13, 6, 7, 14,
      21, 28, 35, 42, 49, 56, 57, 50, 43, 36, 29, 22, 15, 23, 30, 37, 44, 51, 58, 59, 52, 45, 38, 31, 39, 46, 53,
      60, 61, 54, 47, 55, 62, 63]


def test_zigzag_is_the_standard_order():
    assert entropy.ZIGZAG == ZZ and sorted(ZZ) == list(range(64))


def test_block_symbols_by_hand():
    b = np.zeros((2, 64), dtype=np.int64)
    b[0, 0] = 5            # DC 5: category 3
    b[0, ZZ[1]] = -1       # run 0, size 1
    b[0, ZZ[20]] = 3       # run 18 -> ZRL, then run 2, size 2
    b[1, 0] = 5            # DC difference 0: category 0, all-zero AC -> EOB
    dc, ac, amp, n = entropy.plane_histograms(b)
    assert n == 2
    assert dc[3] == 1 and dc[0] == 1 and sum(dc) == 2
    assert ac[0x01] == 1 and ac[0xF0] == 1 and ac[0x22] == 1 and ac[0x00] == 2 and sum(ac) == 5
    assert amp == 3 + 1 + 2


def test_last_coefficient_nonzero_has_no_eob():
    b = np.zeros((1, 64), dtype=np.int64)
    b[0, 63] = 1
    _, ac, _, _ = entropy.plane_histograms(b)
    assert ac[0x00] == 0 and ac[0xF0] == 3 and ac[(14 << 4) | 1] == 1


def test_entropy_bits_closed_forms():
    assert entropy.entropy_bits([4, 4]) == 8.0
    assert entropy.entropy_bits([7]) == 0.0
    assert abs(entropy.entropy_bits([1, 3]) - (2 + 3 * math.log2(4 / 3))) < 1e-12

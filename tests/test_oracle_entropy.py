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


# ---- optimal length-limited prefix code (package-merge) -------------------

import heapq
import itertools


def huffman_cost(counts):
    """Plain Huffman (no length limit), merging the two lightest subtrees:
    the cost is the sum of the merged weights."""
    h = [c for c in counts if c > 0]
    if len(h) < 2:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def huffman_depth(counts):
    h = [(c, 0) for c in counts if c > 0]
    heapq.heapify(h)
    while len(h) > 1:
        (a, da), (b, db) = heapq.heappop(h), heapq.heappop(h)
        heapq.heappush(h, (a + b, max(da, db) + 1))
    return h[0][1]


def brute_force_cost(counts, max_len):
    w = [c for c in counts if c > 0]
    best = None
    for ls in itertools.product(range(1, max_len + 1), repeat=len(w)):
        if sum(2.0 ** -l for l in ls) <= 1.0:
            c = sum(a * b for a, b in zip(w, ls))
            best = c if best is None else min(best, c)
    return best


def test_code_lengths_closed_forms():
    assert entropy.limited_code_lengths([1, 1, 2, 4]) == [3, 3, 2, 1]
    assert entropy.limited_code_lengths([0, 9, 0]) == [0, 1, 0]
    assert entropy.limited_code_lengths([5, 0, 3]) == [1, 0, 1]
    assert entropy.limited_code_lengths([0, 0]) == [0, 0]
    assert entropy.limited_code_lengths([1] * 8) == [3] * 8


def test_code_matches_brute_force_on_small_alphabets():
    rng = np.random.default_rng(7)
    for n in range(2, 7):
        for max_len in (n - 1, 3, 4):
            if (1 << max_len) < n:
                continue
            for _ in range(6):
                c = [int(v) for v in rng.integers(1, 60, size=n)]
                if _ == 0:
                    c = [2 ** k for k in range(n)]      # skewed: the limit binds
                assert entropy.code_cost(c, max_len) == brute_force_cost(c, max_len), (c, max_len)


def test_code_equals_huffman_when_the_limit_is_slack():
    rng = np.random.default_rng(8)
    for _ in range(20):
        c = [int(v) for v in rng.integers(200, 5000, size=256)]
        c[rng.integers(0, 256)] = 0
        assert huffman_depth(c) <= 16
        assert entropy.code_cost(c) == huffman_cost(c)
        ls = entropy.limited_code_lengths(c)
        assert sum(2.0 ** -l for l in ls if l) == 1.0


def test_code_limit_binds_on_fibonacci_weights():
    fib = [1, 1]
    while len(fib) < 24:
        fib.append(fib[-1] + fib[-2])
    assert huffman_depth(fib) == 23
    ls = entropy.limited_code_lengths(fib)
    assert max(ls) == 16 and sum(2.0 ** -l for l in ls) == 1.0
    assert entropy.code_cost(fib) > huffman_cost(fib)
    # within the entropy bound of any prefix code
    n = sum(fib)
    assert entropy.code_cost(fib) >= entropy.entropy_bits(fib) - 1e-9 * n

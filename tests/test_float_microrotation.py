"""The forward kernels run CORDIC micro-rotations 2..N (Sec. 2.5.2) as one
float32 fused multiply-add with directed rounding per half micro-rotation,
on values biased into the range [2^23, 2^24) where every float32 is an
integer.  These checks, on the CPU, re-derive that form from IEEE-754
float32 rounding written out here with exact rationals, read the bias
table the kernels compile with, and compare the result with the oracle's
integer micro-rotations: the rotation blocks alone on random and extreme
inputs, and whole forward 2-D transforms with the oracle's flow graph
running the float form.  They also pin the node bound the kernels' bias
schedule assumes to the oracle's interval propagation."""
import os
import re
import struct
from fractions import Fraction

import numpy as np
import pytest

from oracle import cordic_loeffler as cl
from oracle import codec, interval

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1306_1373_gb300", "csrc", "cordic_loeffler.cuh")
NS = (3, 4, 5, 6)


def header_constants():
    text = open(HDR).read()
    unit = int(re.search(r"kFltUnit = 1LL << (\d+);", text).group(1))
    bound = int(re.search(r"kFwdNodeBound = 1LL << (\d+);", text).group(1))
    vals = {}
    for name, k in re.findall(r"(kFlt\w+[AB]) = (-?\d+) \* kFltUnit", text):
        vals[name] = int(k) << unit if int(k) >= 0 else -((-int(k)) << unit)
    return {"odd_upper": (vals["kFltOddUpperA"], vals["kFltOddUpperB"]),
            "odd_lower": (vals["kFltOddLowerA"], vals["kFltOddLowerB"]),
            "even": (vals["kFltEvenA"], vals["kFltEvenB"])}, 1 << bound


BIASES, NODE_BOUND = header_constants()


def round_f32(r, mode):
    """IEEE-754 binary32 rounding of the exact rational r toward -inf
    ('down') or +inf ('up'); normal range only."""
    r = Fraction(r)
    if r == 0:
        return Fraction(0)
    neg = r < 0
    m = -r if neg else r
    e = m.numerator.bit_length() - m.denominator.bit_length()
    if Fraction(2) ** e > m:
        e -= 1
    assert -126 <= e <= 127
    ulp = Fraction(2) ** (e - 23)
    k = m / ulp
    toward_zero = (mode == "down") != neg          # magnitude rounds down
    kk = k.numerator // k.denominator if toward_zero else -((-k.numerator) // k.denominator)
    v = kk * ulp
    return -v if neg else v


def f32_bits(x):
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def enc(alpha, v):
    """The kernels' bit image of the float alpha + v, as a float value."""
    bits = (0x4A800000 + alpha + v) if alpha > 0 else (0xCA800000 - alpha - v)
    bits &= 0xFFFFFFFF
    x = struct.unpack("<f", struct.pack("<I", bits))[0]
    assert Fraction(x) == alpha + v, (alpha, v)        # the image is exact
    return Fraction(x)


def bias_after(sig, a0, b0, upto):
    a, b = a0, b0
    for i in range(2, upto):
        da, db = Fraction(b, 1 << i), Fraction(a, 1 << i)
        assert da.denominator == 1 and db.denominator == 1
        if sig[i - 1] > 0:
            a, b = a + int(da), b - int(db)
        else:
            a, b = a - int(da), b + int(db)
    return a, b


def rotate_float_form(a, b, sig, biases):
    """One rotation block as the forward kernels compute it."""
    n = len(sig)
    if sig[0] > 0:
        a1, b1 = a + (b >> 1), b - (a >> 1)
    else:
        a1, b1 = a - (b >> 1), b + (a >> 1)
    fa, fb = enc(biases[0], a1), enc(biases[1], b1)
    for i in range(2, n + 1):
        sc = Fraction(1, 1 << i)
        if sig[i - 1] > 0:
            fa, fb = round_f32(fb * sc + fa, "down"), round_f32(-fa * sc + fb, "up")
        else:
            fa, fb = round_f32(-fb * sc + fa, "up"), round_f32(fa * sc + fb, "down")
    ea, eb = bias_after(sig, biases[0], biases[1], n + 1)
    ra, rb = fa - ea, fb - eb
    assert ra.denominator == 1 and rb.denominator == 1
    return int(ra), int(rb)


def max_abs_path(a, b, sig):
    m = max(abs(a), abs(b))
    for i, s in enumerate(sig, start=1):
        if s > 0:
            a, b = a + (b >> i), b - (a >> i)
        else:
            a, b = a - (b >> i), b + (a >> i)
        m = max(m, abs(a), abs(b))
    return m


@pytest.mark.parametrize("n", NS)
def test_forward_node_bound_holds_at_n(n):
    row_max, col_max, _ = interval.forward_bounds(sig=cl.Sigmas(n))
    assert row_max < NODE_BOUND and col_max < NODE_BOUND


def test_bit_image_formula_on_both_signs():
    for alpha in (13 << 20, -(13 << 20), 9 << 20, -(15 << 20)):
        for v in (-(1 << 20), -1, 0, 1, 12345, 1 << 20):
            x = float(alpha + v)
            want = f32_bits(x)
            got = ((0x4A800000 + alpha + v) if alpha > 0 else (0xCA800000 - alpha - v)) & 0xFFFFFFFF
            assert got == want, (alpha, v)


def test_directed_rounding_emulation_against_known_values():
    assert round_f32(Fraction(3, 2), "down") == 1 + Fraction(1, 2)       # exact
    assert round_f32(Fraction((1 << 23) + 1, 2), "down") == Fraction((1 << 23) + 1, 2)
    assert round_f32(Fraction((1 << 24) + 1), "down") == 1 << 24         # ulp 2 above 2^24
    assert round_f32(Fraction((1 << 24) + 1), "up") == (1 << 24) + 2
    assert round_f32(Fraction(-(1 << 24) - 1), "down") == -(1 << 24) - 2
    assert round_f32(Fraction(7, 3), "up") > Fraction(7, 3) > round_f32(Fraction(7, 3), "down")


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("block", ["odd_upper", "odd_lower", "even"])
def test_rotation_block_float_form_equals_integer_form(n, block):
    sig = getattr(cl.Sigmas(n), block)
    rng = np.random.default_rng(100 * n + len(block))
    lim = NODE_BOUND // 2                    # inputs whose whole path stays inside the bound
    pairs = [(int(a), int(b)) for a, b in rng.integers(-lim, lim + 1, size=(1500, 2))]
    pairs += [(int(a), int(b)) for a, b in rng.integers(-64, 65, size=(300, 2))]
    for a in (-lim, -lim + 1, -1, 0, 1, lim - 1, lim):
        for b in (-lim, -lim + 1, -1, 0, 1, lim - 1, lim):
            pairs.append((a, b))
    checked = 0
    for a, b in pairs:
        if max_abs_path(a, b, sig) >= NODE_BOUND:
            continue
        assert rotate_float_form(a, b, sig, BIASES[block]) == cl.cordic_rotate(a, b, sig), (n, block, a, b)
        checked += 1
    assert checked > 1500


@pytest.mark.parametrize("n", NS)
def test_forward_transform_with_float_form_matches_oracle(n, monkeypatch):
    """The oracle's own flow graph, with every forward rotation block run in
    the float form, on random, extreme and structured blocks."""
    sg = cl.Sigmas(n)
    rng = np.random.default_rng(7 + n)
    blocks = [rng.integers(0, 256, size=(8, 8)) for _ in range(25)]
    blocks += [np.full((8, 8), v) for v in (0, 255)]
    ii, jj = np.mgrid[0:8, 0:8]
    blocks += [np.where((ii + jj) % 2, 255, 0), np.where(ii < 4, 0, 255), np.where(jj % 2, 0, 255)]
    for u in range(8):                       # signs of each cosine basis: the extreme column inputs
        for v in range(8):
            basis = np.cos((2 * ii + 1) * u * np.pi / 16) * np.cos((2 * jj + 1) * v * np.pi / 16)
            blocks.append(np.where(basis >= 0, 255, 0))
            blocks.append(np.where(basis >= 0, 0, 255))
    x = np.stack(blocks).astype(np.int64)
    want = codec.forward_coefficients(x, n)
    table = {id(sg.odd_upper): "odd_upper", id(sg.odd_lower): "odd_lower", id(sg.even): "even"}
    plain = cl.cordic_rotate

    def float_form(a, b, sig):
        name = table.get(id(sig))
        if name is None:                     # a Sigmas object built elsewhere: match by value
            for k in ("odd_upper", "odd_lower", "even"):
                if tuple(getattr(sg, k)) == tuple(sig):
                    name = k
        if isinstance(a, (int, np.integer)):
            return rotate_float_form(int(a), int(b), sig, BIASES[name])
        out_a, out_b = np.empty_like(a), np.empty_like(b)
        for idx in np.ndindex(a.shape):
            out_a[idx], out_b[idx] = rotate_float_form(int(a[idx]), int(b[idx]), sig, BIASES[name])
        return out_a, out_b

    monkeypatch.setattr(cl, "cordic_rotate", float_form)
    got = codec.forward_coefficients(x, n)
    monkeypatch.setattr(cl, "cordic_rotate", plain)
    assert np.array_equal(got, want)

"""The kernels quantise 60 of the 64 entries with the plain high word of
Y M + 2^31 instead of the sign-aware definition q = sgn(Y)((|Y| M + 2^31)
>> 32).  These checks prove, with the oracle's own tables and bounds, that
the two agree on every value the forward graph can produce, and that the
four remaining entries (u, v in {0, 4}) do need the sign term."""
import numpy as np
import pytest

from oracle import codec, interval

TIE_ENTRIES = {(0, 0), (0, 4), (4, 0), (4, 4)}
Y_BOUND = 1 << 20


def definition(y, m):
    a = np.abs(y)
    return np.sign(y) * ((a * m + (1 << 31)) >> 32)


def plain_high_word(y, m):
    return (y * m + (1 << 31)) >> 32


def trailing_zeros(m):
    m = int(m)
    return (m & -m).bit_length() - 1


def test_forward_outputs_stay_below_2_pow_20():
    _, col_max, _ = interval.forward_bounds()
    assert col_max < Y_BOUND


def test_non_tie_multipliers_have_at_most_11_trailing_zeros():
    for q in range(1, 256):
        m = codec.quant_multipliers(np.full(64, q))
        for u in range(8):
            for v in range(8):
                if (u, v) not in TIE_ENTRIES:
                    assert trailing_zeros(m[u, v]) <= 11, (u, v, q)


def test_plain_high_word_equals_definition_away_from_tie_entries():
    rng = np.random.default_rng(0)
    y = np.concatenate([np.arange(-4096, 4097), rng.integers(-Y_BOUND, Y_BOUND, 200_000)]).astype(np.int64)
    for q in (1, 2, 3, 7, 16, 50, 99, 128, 255):
        m = codec.quant_multipliers(np.full(64, q))
        for u in range(8):
            for v in range(8):
                if (u, v) in TIE_ENTRIES:
                    continue
                mm = np.int64(m[u, v])
                assert np.array_equal(plain_high_word(y, mm), definition(y, mm)), (u, v, q)


@pytest.mark.parametrize("q", [1, 16, 64])
def test_tie_entries_need_the_sign_term(q):
    m = np.int64(codec.quant_multipliers(np.full(64, q))[0, 0])
    k = trailing_zeros(m)
    y = -np.int64(1 << (31 - k))            # an exact tie: |y| M = 2^31 (mod 2^32)
    assert plain_high_word(y, m) != definition(y, m)
    assert (y * m + (1 << 31) - 1) >> 32 == definition(y, m)   # the sign-aware form the kernels use there

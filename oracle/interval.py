"""Interval propagation through every node of the fixed-point flow graphs.

Proves that the int32 word width of the fixed-point reading of Sec. 2.5.2
is enough: the forward graph is run on intervals covering every level-
shifted input, the inverse graph on intervals covering every clamped
dequantised input, and every value that any +, -, unary minus or >> creates
is recorded.  Floor shifts are monotone, so the interval bounds are sound
(conservative: correlations between nodes are ignored).

Test infrastructure only (see the package docstring).
"""
import numpy as np

from . import spec
from .codec import dequant_weights
from .cordic_loeffler import Sigmas, loeffler8_forward, loeffler8_inverse


class Tracker:
    def __init__(self):
        self.max_abs = 0
        self.nodes = 0

    def see(self, iv):
        self.nodes += 1
        self.max_abs = max(self.max_abs, abs(iv.lo), abs(iv.hi))


class Interval:
    __slots__ = ("lo", "hi", "tr")

    def __init__(self, lo, hi, tr):
        assert lo <= hi
        self.lo, self.hi, self.tr = int(lo), int(hi), tr
        tr.see(self)

    def __add__(self, o):
        return Interval(self.lo + o.lo, self.hi + o.hi, self.tr)

    def __sub__(self, o):
        return Interval(self.lo - o.hi, self.hi - o.lo, self.tr)

    def __neg__(self):
        return Interval(-self.hi, -self.lo, self.tr)

    def __rshift__(self, k):
        return Interval(self.lo >> k, self.hi >> k, self.tr)

    def hull(self, o):
        return Interval(min(self.lo, o.lo), max(self.hi, o.hi), self.tr)


def forward_bounds(p=None, sig=None):
    """Run the forward 2-D transform on intervals.  Returns
    (max |node| in the row pass, max |node| in the column pass, per-output
    (lo, hi) of the column pass as an 8x8 list)."""
    p = spec.P if p is None else p
    sig = Sigmas() if sig is None else sig
    lo, hi = -128 * (1 << p), 127 * (1 << p)
    tr1 = Tracker()
    row_out = loeffler8_forward([Interval(lo, hi, tr1) for _ in range(8)], sig)
    tr2 = Tracker()
    # every row has the same input interval, so column v sees row_out[v] 8 times
    out = [[None] * 8 for _ in range(8)]
    for v in range(8):
        col_in = [Interval(row_out[v].lo, row_out[v].hi, tr2) for _ in range(8)]
        col_out = loeffler8_forward(col_in, sig)
        for u in range(8):
            out[u][v] = (col_out[u].lo, col_out[u].hi)
    return tr1.max_abs, tr2.max_abs, out


def inverse_bounds(dc_offset=0, sig=None, n=None):
    """Run the inverse 2-D transform on the intervals the dequantiser can
    produce (|clamp(qQ)| <= 4096 times W_uv).  ``dc_offset`` adds a constant
    to the (0, 0) input, covering implementations that fold the descale
    rounding term into the DC coefficient.  n: CORDIC micro-rotations per
    rotation (None: the spec's).  Returns (max |node| in the column pass,
    max |node| in the row pass)."""
    sig = Sigmas(n) if sig is None else sig
    w = dequant_weights(n)
    tr1 = Tracker()
    cols = []
    for v in range(8):
        col_in = []
        for u in range(8):
            b = spec.DQ_CLAMP * int(w[u, v])
            off = dc_offset if (u == 0 and v == 0) else 0
            col_in.append(Interval(-b + off, b + off, tr1))
        cols.append(loeffler8_inverse(col_in, sig))
    tr2 = Tracker()
    for i in range(8):
        row_in = [Interval(cols[v][i].lo, cols[v][i].hi, tr2) for v in range(8)]
        loeffler8_inverse(row_in, sig)
    return tr1.max_abs, tr2.max_abs


def worst_case_product_bits(y_bound, qtab_min=1, n=None):
    """Bits needed by |Y| * M + 2^31 in the quantiser for the largest M."""
    from .codec import quant_multipliers
    m = int(np.max(quant_multipliers(np.full((8, 8), qtab_min), n)))
    return (y_bound * m + (1 << 31)).bit_length(), m

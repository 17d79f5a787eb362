"""Linear (untruncated) model of the Cordic-Loeffler flow graph and a
rigorous bound on the fixed-point coefficient error.

Running the flow graph of ``cordic_loeffler`` on ``Exact`` values, whose
">> i" is an exact division by 2^i, gives the linear map A_N of the graph
(CORDIC rotations by the achieved angles, times their gain).  Running it on
``ErrInterval`` values tracks how far the floor shifts can move each node
from that linear map: a floor shift of an integer v by i differs from
v / 2^i by a value in [-(1 - 2^-i), 0].

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np

from . import spec
from .cordic_loeffler import Sigmas, gains, loeffler8_forward, loeffler8_inverse
from .exact_dct import dct_matrix


class Exact:
    """A real number whose >> is exact division by a power of two."""
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = v

    def __add__(self, o):
        return Exact(self.v + o.v)

    def __sub__(self, o):
        return Exact(self.v - o.v)

    def __neg__(self):
        return Exact(-self.v)

    def __rshift__(self, k):
        return Exact(self.v / float(1 << k))


def graph_matrix(fn, sig):
    """Matrix of the linear model of an 8-point graph: column j is the image
    of the j-th unit vector."""
    a = np.zeros((8, 8))
    for j in range(8):
        e = [Exact(1.0 if k == j else 0.0) for k in range(8)]
        out = fn(e, sig)
        a[:, j] = [o.v for o in out]
    return a


def forward_matrix(n=None):
    n = spec.N if n is None else n
    return graph_matrix(loeffler8_forward, Sigmas(n))


def inverse_matrix(n=None):
    n = spec.N if n is None else n
    return graph_matrix(loeffler8_inverse, Sigmas(n))


def normalised_forward(n=None):
    """diag(1 / (sqrt8 g)) A_N: the orthonormal transform the graph realises."""
    g = np.array(gains(n))
    return forward_matrix(n) / (math.sqrt(8.0) * g)[:, None]


class ErrInterval:
    """Interval of the deviation of a node from the linear model."""
    __slots__ = ("lo", "hi")

    def __init__(self, lo, hi):
        self.lo, self.hi = float(lo), float(hi)

    def __add__(self, o):
        return ErrInterval(self.lo + o.lo, self.hi + o.hi)

    def __sub__(self, o):
        return ErrInterval(self.lo - o.hi, self.hi - o.lo)

    def __neg__(self):
        return ErrInterval(-self.hi, -self.lo)

    def __rshift__(self, k):
        s = float(1 << k)
        return ErrInterval(self.lo / s - (1.0 - 1.0 / s), self.hi / s)

    @property
    def mag(self):
        return max(abs(self.lo), abs(self.hi))


def forward_truncation_bound(n=None):
    """Per-coefficient bound (8x8, in units of Y) of |Y_fixed - A2 x| for the
    2-D forward transform (row pass then column pass)."""
    sig = Sigmas(spec.N if n is None else n)
    zero = [ErrInterval(0.0, 0.0) for _ in range(8)]
    row_err = loeffler8_forward(zero, sig)          # the same for every row
    out = np.zeros((8, 8))
    for v in range(8):
        col_in = [ErrInterval(row_err[v].lo, row_err[v].hi) for _ in range(8)]
        col_err = loeffler8_forward(col_in, sig)
        for u in range(8):
            out[u, v] = col_err[u].mag
    return out


def cordic_vs_exact_bound(n=None, p=None):
    """Bound on |X_cordic(u, v) - X_exact(u, v)| on the orthonormal scale for
    any 8x8 block of level-shifted pixels in [-128, 127], where
    X_cordic = Y / (8 2^P g_u g_v).  Sum of the linear-model part
    128 * sum_ij |Cn(u,i) Cn(v,j) - C(u,i) C(v,j)| and the truncation part."""
    n = spec.N if n is None else n
    p = spec.P if p is None else p
    cn = normalised_forward(n)
    c = dct_matrix(8)
    g = np.array(gains(n))
    lin = np.zeros((8, 8))
    for u in range(8):
        for v in range(8):
            lin[u, v] = 128.0 * np.abs(np.outer(cn[u], cn[v]) - np.outer(c[u], c[v])).sum()
    trunc = forward_truncation_bound(n) / (8.0 * (1 << p) * np.outer(g, g))
    return lin + trunc

"""Fixed-point Cordic-based Loeffler 8-point DCT and its transpose (inverse).

Sec. 2.5.2 describes the Loeffler flow graph: four stages executed in
series; stage 2 splits the data into an even part and an odd part; the even
part is a 4-point DCT that stage 3 splits again; the Cordic-based variant
replaces the plane rotations of the flow graph by CORDIC rotation blocks
and applies the sqrt(2) scalings ("rotating ... by pi/4", stage 4).  Fig. 1
(the flow graph itself) is missing from the text, so the graph below is the
standard Loeffler graph, written out:

  stage 1   s_n = x_n + x_{7-n},  d_n = x_n - x_{7-n}        (n = 0..3)
  stage 2   even: e0 = s0 + s3, e3 = s0 - s3, e1 = s1 + s2, e2 = s1 - s2
            odd:  (a4, a7) = rot(d3, d0, 3pi/16), (a5, a6) = rot(d2, d1, pi/16)
  stage 3   even: Y0 = e0 + e1, Y4 = e0 - e1, (Y2, Y6) = sqrt2 * rot(e2, e3, 3pi/8)
            odd:  b4 = a4 + a6, b6 = a4 - a6, b7 = a7 + a5, b5 = a7 - a5
  stage 4   Y1 = b7 + b4, Y7 = b7 - b4, Y3 = sqrt2 * b5, Y5 = sqrt2 * b6

with rot(a, b, t) = (a cos t + b sin t, -a sin t + b cos t).  With exact
rotations Y = sqrt(8) * (orthonormal DCT-II of x) (checked by the tests).

Fixed-point reading (all numbers come from the spec file):
* every rot() is a CORDIC rotation of N micro-rotations with shifts
  i = 1..N; micro-rotation i maps (a, b) to (a + s_i (b >> i), b - s_i (a >> i))
  using the values from before the step, with ">>" an arithmetic (floor)
  shift and s_i = +-1 from the greedy rule on atan(2^-i);
* 3pi/8 is a quarter turn (a, b) -> (b, -a) followed by a CORDIC rotation
  of -pi/8;
* the three sqrt(2) factors and the CORDIC gain K_N are not computed; they
  are folded into the quantiser and dequantiser tables (``codec``).

The inverse is the transposed flow graph: each step replaced by its
transpose in reverse order; a micro-rotation's transpose is the same
micro-rotation with -s_i, applied in ascending i; the quarter turn's
transpose is (a, b) -> (-b, a).

The functions only use +, -, unary minus and >> on their values, so they
run unchanged on numpy integer arrays and on ``oracle.interval.Interval``.

Test infrastructure only (see the package docstring).
"""
import math

from . import spec


def cordic_sigmas(angle, n):
    """Greedy CORDIC direction choice: z = angle; for i = 1..n take
    s_i = +1 if z >= 0 else -1 and subtract s_i * atan(2^-i) from z."""
    z = float(angle)
    sig = []
    for i in range(1, n + 1):
        s = 1 if z >= 0.0 else -1
        sig.append(s)
        z -= s * math.atan(2.0 ** (-i))
    return tuple(sig)


def cordic_residual(angle, sig):
    """Angle left over after the micro-rotations of ``sig`` (radians)."""
    z = float(angle)
    for i, s in enumerate(sig, start=1):
        z -= s * math.atan(2.0 ** (-i))
    return z


def cordic_gain(n):
    """K_n = prod_{i=1..n} sqrt(1 + 4^-i): the length growth of n micro-rotations."""
    k = 1.0
    for i in range(1, n + 1):
        k *= math.sqrt(1.0 + math.ldexp(1.0, -2 * i))
    return k


class Sigmas:
    """The three direction tables of one flow graph."""

    def __init__(self, n=None):
        n = spec.N if n is None else n
        self.n = n
        self.odd_upper = cordic_sigmas(spec.ANGLE_ODD_UPPER * math.pi, n)   # rot(d3, d0, 3pi/16)
        self.odd_lower = cordic_sigmas(spec.ANGLE_ODD_LOWER * math.pi, n)   # rot(d2, d1, pi/16)
        self.even = cordic_sigmas(spec.ANGLE_EVEN_CORDIC * math.pi, n)      # rot(., ., -pi/8)


def cordic_rotate(a, b, sig):
    """Forward CORDIC rotation: micro-rotations i = 1..N in ascending order."""
    for i, s in enumerate(sig, start=1):
        if s > 0:
            a, b = a + (b >> i), b - (a >> i)
        else:
            a, b = a - (b >> i), b + (a >> i)
    return a, b


def cordic_rotate_t(a, b, sig):
    """Transposed CORDIC rotation: the same shifts with -s_i, ascending i."""
    for i, s in enumerate(sig, start=1):
        if s > 0:
            a, b = a - (b >> i), b + (a >> i)
        else:
            a, b = a + (b >> i), b - (a >> i)
    return a, b


def loeffler8_forward(x, sig):
    """Forward 8-point Cordic-Loeffler flow graph on 8 values; returns
    [Y0..Y7] with Y_k ~ sqrt(8) g_k X_k (g from ``gains``)."""
    # stage 1: butterflies
    s0, s1, s2, s3 = (x[n] + x[7 - n] for n in range(4))
    d0, d1, d2, d3 = (x[n] - x[7 - n] for n in range(4))
    # stage 2, even part: 4-point butterflies
    e0 = s0 + s3
    e3 = s0 - s3
    e1 = s1 + s2
    e2 = s1 - s2
    # stage 2, odd part: two rotation blocks
    a4, a7 = cordic_rotate(d3, d0, sig.odd_upper)
    a5, a6 = cordic_rotate(d2, d1, sig.odd_lower)
    # stage 3, even part: DC/Nyquist butterfly and the 3pi/8 rotation
    y0 = e0 + e1
    y4 = e0 - e1
    y2, y6 = cordic_rotate(e3, -e2, sig.even)      # quarter turn of (e2, e3), then -pi/8
    # stage 3, odd part
    b4 = a4 + a6
    b6 = a4 - a6
    b7 = a7 + a5
    b5 = a7 - a5
    # stage 4 (sqrt2 scalings folded into the tables)
    y1 = b7 + b4
    y7 = b7 - b4
    y3 = b5
    y5 = b6
    return [y0, y1, y2, y3, y4, y5, y6, y7]


def loeffler8_inverse(y, sig):
    """Transpose of ``loeffler8_forward``: the inverse flow graph."""
    # stage 4 transposed
    b7 = y[1] + y[7]
    b4 = y[1] - y[7]
    b5 = y[3]
    b6 = y[5]
    # stage 3 transposed
    a4 = b4 + b6
    a6 = b4 - b6
    a7 = b7 + b5
    a5 = b7 - b5
    e0 = y[0] + y[4]
    e1 = y[0] - y[4]
    p, q = cordic_rotate_t(y[2], y[6], sig.even)
    e2, e3 = -q, p                                 # transposed quarter turn
    # stage 2 transposed
    d3, d0 = cordic_rotate_t(a4, a7, sig.odd_upper)
    d2, d1 = cordic_rotate_t(a5, a6, sig.odd_lower)
    s0 = e0 + e3
    s3 = e0 - e3
    s1 = e1 + e2
    s2 = e1 - e2
    # stage 1 transposed
    return [s0 + d0, s1 + d1, s2 + d2, s3 + d3, s3 - d3, s2 - d2, s1 - d1, s0 - d0]


def gains(n=None):
    """Per-output gain of one pass relative to sqrt(8) * orthonormal DCT:
    g = [1, K, K/sqrt2, K/sqrt2, 1, K/sqrt2, K/sqrt2, K]."""
    n = spec.N if n is None else n
    k = cordic_gain(n)
    kr = k / math.sqrt(2.0)
    return [1.0, k, kr, kr, 1.0, kr, kr, k]

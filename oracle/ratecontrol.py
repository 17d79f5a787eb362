"""Quality search for a target PSNR: the plain pipeline's 8-step bisection
and the learned controller's accept / fall-back rule.

PSNR(q) is that of Eq. 23 with MAX = 255 over all samples of an image (for
4:2:0 frames: the sample-weighted PSNR over the three planes, i.e. one SSE
over all samples).  Every decision is taken on the integer SSE:

  PSNR >= T             <=>  SSE <= floor(65025 n / 10^(T/10))
  |PSNR - T| <= 0.25    <=>  ceil(65025 n / 10^((T+0.25)/10)) <= SSE
                              <= floor(65025 n / 10^((T-0.25)/10))

Bisection (8 steps over the integer qualities 1..100): lo = 1, hi = 100;
mid = (lo + hi) // 2; if PSNR(mid) >= T then hi = mid else lo = mid + 1.
After 7 steps lo = hi; the 8th evaluates that quality.  Q* = min(hi, 100),
the smallest quality meeting the target when PSNR rises with quality; an
image whose PSNR(100) is below the target ends at Q* = 100 and is
"unreachable".  The learned controller predicts a quality, runs the plain
pipeline once and keeps the result when its PSNR is within 0.25 dB of the
target; otherwise it falls back to the bisection.

Test infrastructure only (see the package docstring).
"""
import math

from . import psnr as _psnr

MAX2 = 255.0 * 255.0


def sse_at_most(target_db, n):
    """Largest SSE whose PSNR is >= target_db."""
    return int(math.floor(MAX2 * float(n) / (10.0 ** (float(target_db) / 10.0))))


def sse_band(target_db, n, tol=0.25):
    """(lo, hi) SSE range whose PSNR is within tol dB of the target."""
    lo = int(math.ceil(MAX2 * float(n) / (10.0 ** ((float(target_db) + tol) / 10.0))))
    hi = int(math.floor(MAX2 * float(n) / (10.0 ** ((float(target_db) - tol) / 10.0))))
    return lo, hi


def bisect_quality(sse_of_quality, target_db, n, steps=8):
    """8-step bisection; sse_of_quality(q) -> integer SSE.  Returns
    (Q*, SSE(Q*), list of evaluated qualities)."""
    thr = sse_at_most(target_db, n)
    lo, hi = 1, 100
    seen = []
    last = {}
    for _ in range(steps):
        mid = (lo + hi) // 2
        s = sse_of_quality(mid)
        seen.append(mid)
        last[mid] = s
        if s <= thr:
            hi = mid
        else:
            lo = mid + 1
    q = min(hi, 100)
    s = last[q] if q in last else sse_of_quality(q)
    return q, s, seen


def learned_decision(sse_pred, target_db, n, tol=0.25):
    """True when the prediction's SSE puts its PSNR within tol of the target."""
    lo, hi = sse_band(target_db, n, tol)
    return lo <= sse_pred <= hi


def psnr(sse, n):
    return _psnr.psnr_from_sse(int(sse), int(n))

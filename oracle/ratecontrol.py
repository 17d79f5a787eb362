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
the smallest quality meeting the target when PSNR rises with quality.

Band pick (the controller's goal is a final PSNR within 0.25 dB of the
target, either way): when PSNR(Q*) lies outside that band but the last
quality the bisection rejected lies inside it, that quality is the result.
lo only moves on a rejection (to mid + 1), so the last rejected quality is
Q* - 1 whenever any step rejected.

Out-of-band results are split by the two evaluations around the answer:
"unreachable" when they show that no quality lands in the band as long as
PSNR rises with quality (PSNR(100) below T - 0.25, or PSNR(Q*) above
T + 0.25 with Q* = 1 or PSNR(Q* - 1) below T - 0.25), else "missed".

The learned controller predicts a quality, runs the plain pipeline once and
keeps the result when its PSNR is within 0.25 dB of the target; otherwise it
falls back to the bisection.

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


def bisect_quality(sse_of_quality, target_db, n, steps=8, band_tol=None):
    """8-step bisection; sse_of_quality(q) -> integer SSE.  Returns
    (quality, its SSE, list of evaluated qualities).  Without band_tol the
    quality is Q*; with it, the band pick described above."""
    thr = sse_at_most(target_db, n)
    lo, hi = 1, 100
    seen = []
    last = {}
    rejected = None
    for _ in range(steps):
        mid = min((lo + hi) // 2, 100)
        s = sse_of_quality(mid)
        seen.append(mid)
        last[mid] = s
        if s <= thr:
            hi = mid
        else:
            lo = mid + 1
            rejected = mid
    q = min(hi, 100)
    s = last[q] if q in last else sse_of_quality(q)
    if band_tol is not None and rejected is not None:
        blo, bhi = sse_band(target_db, n, band_tol)
        if not (blo <= s <= bhi) and blo <= last[rejected] <= bhi:
            return rejected, last[rejected], seen
    return q, s, seen


def band_outcome(q, sse_q, q_below, sse_below, target_db, n, tol=0.25):
    """'within', 'unreachable' or 'missed' for a final quality q with SSE
    sse_q, given the evaluated quality below it (q_below, its SSE; q_below
    None or != q - 1 when it was not evaluated)."""
    blo, bhi = sse_band(target_db, n, tol)
    if blo <= sse_q <= bhi:
        return "within"
    if sse_q > bhi and q == 100:
        return "unreachable"                      # even quality 100 is too lossy
    if sse_q < blo and (q == 1 or (q_below == q - 1 and sse_below > bhi)):
        return "unreachable"                      # the band falls between q - 1 and q
    return "missed"


def learned_decision(sse_pred, target_db, n, tol=0.25):
    """True when the prediction's SSE puts its PSNR within tol of the target."""
    lo, hi = sse_band(target_db, n, tol)
    return lo <= sse_pred <= hi


def psnr(sse, n):
    return _psnr.psnr_from_sse(int(sse), int(n))

"""Sum of squared errors and PSNR (Eq. 23, Eq. 24).

Eq. 24: MSE = (1 / (N M)) sum_i sum_j (O(i, j) - C(i, j))^2.
Eq. 23: PSNR = 20 log10(MAX / sqrt(MSE)), written here as
10 log10(MAX^2 * n / SSE), the same value.  The text says MAX is the largest
pixel value of the original O; the default reading is the largest value an
8-bit sample can take (255), and ``max_of_original`` gives the literal one.

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np

from . import spec


def sse(original, reconstruction):
    """Exact integer sum of squared differences (Python int)."""
    d = np.asarray(original, dtype=np.int64) - np.asarray(reconstruction, dtype=np.int64)
    return int((d * d).sum())


def psnr_from_sse(total_sse, n_samples, max_value=None):
    """PSNR in dB from an integer SSE over n samples; +inf when SSE is 0."""
    mx = spec.MAX_DEFAULT if max_value is None else max_value
    if total_sse == 0:
        return math.inf
    return 10.0 * math.log10(float(mx) * float(mx) * float(n_samples) / float(total_sse))


def psnr(original, reconstruction, max_of_original=False):
    o = np.asarray(original)
    mx = int(o.max()) if max_of_original else None
    return psnr_from_sse(sse(o, reconstruction), o.size, mx)


def psnr_eq23(original, reconstruction, max_value=255.0):
    """Eq. 23 and Eq. 24 evaluated literally in FP64 (mean, sqrt, 20 log10)."""
    o = np.asarray(original, dtype=np.float64)
    c = np.asarray(reconstruction, dtype=np.float64)
    mse = np.mean((o - c) ** 2)
    if mse == 0.0:
        return math.inf
    return 20.0 * math.log10(max_value / math.sqrt(mse))

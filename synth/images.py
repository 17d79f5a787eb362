"""Seeded synthetic images standing in for the paper's test photographs.

The paper measures on grayscale photographs (Lena, Cable-car) at sizes from
200x200 to 3072x3072 (Tables 1 and 2); those images are not available, so
every workload here is generated from a seed:

* ``sinusoid_image``: a sum of random 2-D sinusoids (periods log-uniform in
  [4, 128] px, orientation uniform in [0, pi), phase uniform in [0, 2 pi)),
  min-max scaled to [0, 255], plus Gaussian noise, rounded and clipped.
* ``powerlaw_image``: 1/f^beta noise (power spectrum ~ f^-beta, so the
  Fourier amplitude ~ f^(-beta/2)), normalised to mean 128 and std 40, plus
  random half-plane step edges (amplitude +-U(20, 80)) and optional random
  constant rectangles, rounded and clipped.
* ``yuv420_frame``: a power-law luma plane and two half-resolution chroma
  planes (smoother, std 16 around 128).

Everything is generated with torch on the requested device from
``torch.Generator(device).manual_seed(seed)``.  Results on CPU and CUDA
differ (different random streams and FFTs); every comparison therefore feeds
the same uint8 buffer to both sides.
"""
import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    return g


def _uniform(g, device, lo, hi, shape=()):
    return lo + (hi - lo) * torch.rand(shape, generator=g, device=device, dtype=torch.float64)


def _to_u8(x):
    return torch.clamp(torch.round(x), 0, 255).to(torch.uint8)


def sinusoid_image(height, width, seed, n_waves=8, noise_sigma=5.0, device="cpu"):
    """Sum of ``n_waves`` random 2-D sinusoids scaled to [0, 255] plus noise."""
    g = _gen(seed, device)
    yy = torch.arange(height, device=device, dtype=torch.float64).view(-1, 1)
    xx = torch.arange(width, device=device, dtype=torch.float64).view(1, -1)
    acc = torch.zeros(height, width, device=device, dtype=torch.float64)
    for _ in range(n_waves):
        period = math.exp(float(_uniform(g, device, math.log(4.0), math.log(128.0))))
        theta = float(_uniform(g, device, 0.0, math.pi))
        phase = float(_uniform(g, device, 0.0, 2.0 * math.pi))
        k = 2.0 * math.pi / period
        acc += torch.sin(k * (math.cos(theta) * xx + math.sin(theta) * yy) + phase)
    lo, hi = acc.min(), acc.max()
    img = (acc - lo) / torch.clamp(hi - lo, min=1e-12) * 255.0
    img += noise_sigma * torch.randn(height, width, generator=g, device=device, dtype=torch.float64)
    return _to_u8(img)


def _powerlaw_field(height, width, beta, g, device):
    noise = torch.randn(height, width, generator=g, device=device, dtype=torch.float32)
    spec = torch.fft.rfft2(noise)
    fy = torch.fft.fftfreq(height, device=device).view(-1, 1)
    fx = torch.fft.rfftfreq(width, device=device).view(1, -1)
    f = torch.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    amp = f.pow(-beta / 2.0)
    amp[0, 0] = 0.0
    field = torch.fft.irfft2(spec * amp, s=(height, width))
    field = field - field.mean()
    return field / torch.clamp(field.std(), min=1e-12)


def _add_edges(img, k, g, device):
    height, width = img.shape
    yy = torch.arange(height, device=device, dtype=torch.float32).view(-1, 1)
    xx = torch.arange(width, device=device, dtype=torch.float32).view(1, -1)
    for _ in range(k):
        ang = float(_uniform(g, device, 0.0, 2.0 * math.pi))
        x0 = float(_uniform(g, device, 0.0, width))
        y0 = float(_uniform(g, device, 0.0, height))
        amp = float(_uniform(g, device, 20.0, 80.0))
        sign = 1.0 if float(_uniform(g, device, 0.0, 1.0)) < 0.5 else -1.0
        side = (math.cos(ang) * (xx - x0) + math.sin(ang) * (yy - y0)) > 0
        img = img + sign * amp * side.to(img.dtype)
    return img


def _add_rects(img, k, g, device):
    height, width = img.shape
    for _ in range(k):
        w = int(_uniform(g, device, 0.05, 0.5) * width) + 1
        h = int(_uniform(g, device, 0.05, 0.5) * height) + 1
        x0 = int(_uniform(g, device, 0.0, max(width - w, 1)))
        y0 = int(_uniform(g, device, 0.0, max(height - h, 1)))
        level = float(_uniform(g, device, 0.0, 255.0))
        img[y0:y0 + h, x0:x0 + w] = level
    return img


def powerlaw_image(height, width, seed, beta=2.0, edges=True, rects=0, std=40.0,
                   mean=128.0, device="cpu"):
    """1/f^beta noise plus 2..6 random step edges (and ``rects`` rectangles;
    ``rects=-1`` draws 1..8 of them)."""
    g = _gen(seed, device)
    img = mean + std * _powerlaw_field(height, width, beta, g, device)
    if edges:
        k = int(_uniform(g, device, 2.0, 7.0))
        img = _add_edges(img, k, g, device)
    if rects:
        k = int(_uniform(g, device, 1.0, 9.0)) if rects < 0 else int(rects)
        img = _add_rects(img, k, g, device)
    return _to_u8(img)


def yuv420_frame(width, height, seed, beta=2.0, device="cpu"):
    """(Y, Cb, Cr) uint8 planes of a 4:2:0 frame; chroma is ceil(W/2) x ceil(H/2)."""
    cw, ch = (width + 1) // 2, (height + 1) // 2
    y = powerlaw_image(height, width, seed, beta=beta, device=device)
    cb = powerlaw_image(ch, cw, seed * 2 + 1, beta=beta + 0.5, edges=False, std=16.0, device=device)
    cr = powerlaw_image(ch, cw, seed * 2 + 2, beta=beta + 0.5, edges=False, std=16.0, device=device)
    return y, cb, cr


def batch_workload(n=512, seed=2, lo=64, hi=2048):
    """Per-image (width, height, quality, beta) for the batched workload:
    W and H uniform over multiples of 8 in [lo, hi], quality uniform in
    [10, 95], beta uniform in [1, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ws = rng.integers(lo // 8, hi // 8 + 1, size=n) * 8
    hs = rng.integers(lo // 8, hi // 8 + 1, size=n) * 8
    qs = rng.integers(10, 96, size=n)
    bs = rng.uniform(1.0, 3.0, size=n)
    return [dict(width=int(w), height=int(h), quality=int(q), beta=float(b), seed=1000003 * seed + i)
            for i, (w, h, q, b) in enumerate(zip(ws, hs, qs, bs))]


def ratecontrol_workload(n=20000, seed=3, lo=256, hi=1024):
    """Per-image parameters of the learned-rate-control set: W and H
    uniform over multiples of 8 in [lo, hi], beta in [1, 3], a target PSNR
    uniform in [28, 42] dB."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ws = rng.integers(lo // 8, hi // 8 + 1, size=n) * 8
    hs = rng.integers(lo // 8, hi // 8 + 1, size=n) * 8
    bs = rng.uniform(1.0, 3.0, size=n)
    ts = rng.uniform(28.0, 42.0, size=n)
    return [dict(width=int(w), height=int(h), beta=float(b), target=float(t), seed=1000003 * seed + i)
            for i, (w, h, b, t) in enumerate(zip(ws, hs, bs, ts))]


def stream_workload(n=2000, seed=4):
    """Per-frame parameters of the mixed 4:2:0 stream: size from
    {1280x720, 1920x1080, 3840x2160}, target PSNR uniform in [30, 40] dB."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [(1280, 720), (1920, 1080), (3840, 2160)]
    idx = rng.integers(0, 3, size=n)
    bs = rng.uniform(1.0, 3.0, size=n)
    ts = rng.uniform(30.0, 40.0, size=n)
    return [dict(width=sizes[k][0], height=sizes[k][1], beta=float(b), target=float(t),
                 seed=1000003 * seed + i) for i, (k, b, t) in enumerate(zip(idx, bs, ts))]


def ragged_sizes():
    """Small shapes covering full tiles, ragged right/bottom edges and strips."""
    return [(8, 8), (8, 16), (16, 8), (7, 13), (13, 7), (1, 1), (1, 9), (9, 1),
            (8, 264), (264, 8), (37, 29), (61, 300), (540 // 4, 960 // 4)]

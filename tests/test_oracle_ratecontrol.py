"""Pins for the rate controller's oracle: network gradient against finite
differences, GELU and bfloat16 rounding against library routines and
identities, Adam's first step in closed form, the statistics words of
constant blocks, and the bisection against a brute-force scan."""
import math

import numpy as np
import pytest
import torch

from oracle import codec, features, ijg, mlp, psnr, ratecontrol, spec


def rand_batch(seed, b=16):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(b, mlp.N_IN)) * 2.0 + 1.0
    t = rng.uniform(0, 1, size=b)
    return x, t, np.full(mlp.N_IN, 1.0), np.full(mlp.N_IN, 2.0)


def test_param_layout():
    assert mlp.N_PARAMS == 64 * 80 + 64 + 64 * 64 + 64 + 64 + 1 == 9409
    p = np.arange(mlp.N_PARAMS, dtype=np.float64)
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)


def test_gradient_matches_central_differences():
    x, t, mean, std = rand_batch(1)
    p = mlp.init_params(7) + np.random.default_rng(2).normal(0, 0.05, mlp.N_PARAMS)
    loss, g = mlp.loss_and_grad(p, x, t, mean, std, mode="fp32")
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [9408, 9344, 5120, 0]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, x, t, mean, std, mode="fp32")
        lm, _ = mlp.loss_and_grad(p - e, x, t, mean, std, mode="fp32")
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_gelu_identities_and_derivative():
    a = np.linspace(-6, 6, 241)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(a) - mlp.gelu(-a), a, atol=1e-14)          # x Phi(x) - (-x) Phi(-x) = x
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    h = 1e-6
    fd = (mlp.gelu(a + h) - mlp.gelu(a - h)) / (2 * h)
    assert np.allclose(fd, mlp.gelu_grad(a), atol=1e-8)
    # Phi(1) from the textbook value 0.8413447460685429
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(0, 3, 5000), [0.0, -0.0, 1.0, 1.00390625, 1.001953125, 65504.0, -3.14159]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    newp, m, v = mlp.adam_step(p, np.zeros(3), np.zeros(3), g, step=1, lr=0.01)
    # m_hat = g, v_hat = g^2: the first step moves each parameter by lr * g / (|g| + eps)
    assert np.allclose(newp, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_reduces_loss_on_a_learnable_map():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(256, mlp.N_IN))
    t = 1.0 / (1.0 + np.exp(-(x[:, 0] - 0.5 * x[:, 3])))
    mean, std = np.zeros(mlp.N_IN), np.ones(mlp.N_IN)
    p = mlp.init_params(1)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0, _ = mlp.loss_and_grad(p, x, t, mean, std, "fp32")
    for k in range(1, 201):
        _, g = mlp.loss_and_grad(p, x, t, mean, std, "fp32")
        p, m, v = mlp.adam_step(p, m, v, g, k, lr=3e-3)
    l1, _ = mlp.loss_and_grad(p, x, t, mean, std, "fp32")
    assert l1 < 0.1 * l0


@pytest.mark.parametrize("c", [0, 37, 128, 200, 255])
def test_statistics_of_constant_block(c):
    st = features.block_stats(np.full((3, 8, 8), c, dtype=np.uint8))
    dc = (abs(64 * (c - 128) * (1 << spec.P)) >> (spec.P + 1)) ** 2
    assert st[0] == 3 * dc and sum(st[1:64]) == 0
    assert st[64] == 3 * 64 * c and st[65] == 3 * 64 * c * c
    assert st[66] == c and st[67] == c
    assert st[68:72] == [0, 0, 0, 0]
    assert st[72:76] == [3, 3, 3, 3]
    assert st[76] == 3 and st[77] == 192


def test_statistics_gradients_bruteforce():
    rng = np.random.default_rng(6)
    b = rng.integers(0, 256, size=(2, 8, 8)).astype(np.uint8)
    st = features.block_stats(b)
    adx = sum(abs(int(b[k, r, c + 1]) - int(b[k, r, c])) for k in range(2) for r in range(8) for c in range(7))
    dy2 = sum((int(b[k, r + 1, c]) - int(b[k, r, c])) ** 2 for k in range(2) for r in range(7) for c in range(8))
    assert st[68] == adx and st[71] == dy2


def test_features_shape_and_bias():
    img = np.random.default_rng(7).integers(0, 256, size=(40, 56)).astype(np.uint8)
    st = features.plane_stats(img)
    f = features.features_from_stats(st, 56, 40, 35.0)
    assert f.shape == (80,) and f[79] == 1.0 and f[78] == 0.0
    assert abs(f[76] - math.log2(56) / 11) < 1e-15


def test_sse_thresholds():
    for n in (64, 1000, 262144):
        for t in (28.0, 33.3, 42.0):
            s = ratecontrol.sse_at_most(t, n)
            assert psnr.psnr_from_sse(s, n) >= t
            assert psnr.psnr_from_sse(s + 1, n) < t
            lo, hi = ratecontrol.sse_band(t, n)
            assert abs(psnr.psnr_from_sse(hi, n) - t) <= 0.25 and psnr.psnr_from_sse(hi + 1, n) < t - 0.25
            assert lo == 0 or (abs(psnr.psnr_from_sse(lo, n) - t) <= 0.25 and psnr.psnr_from_sse(lo - 1, n) > t + 0.25)


def _sse_curve(img):
    out = {}
    for q in range(1, 101):
        Q = ijg.luma_table(q)
        r = codec.reconstruct_plane(codec.compress_plane(img, Q), Q, *img.shape)
        out[q] = psnr.sse(img, r)
    return out


def test_bisection_equals_bruteforce_scan():
    from synth import powerlaw_image
    img = powerlaw_image(48, 64, seed=8).numpy()
    curve = _sse_curve(img)
    n = img.size
    for t in np.linspace(24.0, 48.0, 25):
        q, s, seen = ratecontrol.bisect_quality(curve.__getitem__, t, n)
        assert len(seen) == 8 and s == curve[q]
        thr = ratecontrol.sse_at_most(t, n)
        ok = [k for k in range(1, 101) if curve[k] <= thr]
        if not ok:
            assert q == 100                      # unreachable target
        else:
            # bisection finds a quality meeting the target whose predecessor fails
            assert curve[q] <= thr and (q == 1 or curve[q - 1] > thr)
            if all(curve[k + 1] <= curve[k] for k in range(1, 100)):
                assert q == min(ok)


def test_bisection_extremes():
    q, _, _ = ratecontrol.bisect_quality(lambda k: 0, 60.0, 100)
    assert q == 1
    q, _, _ = ratecontrol.bisect_quality(lambda k: 10 ** 9, 20.0, 100)
    assert q == 100


def _band_quals(curve, t, n, tol=0.25):
    lo, hi = ratecontrol.sse_band(t, n, tol)
    return [k for k in range(1, 101) if lo <= curve[k] <= hi]


def _outcome_of(curve, t, n):
    q, s, seen = ratecontrol.bisect_quality(curve.__getitem__, t, n, band_tol=0.25)
    qs, _, _ = ratecontrol.bisect_quality(curve.__getitem__, t, n)
    below = qs - 1 if (qs - 1) in seen else None
    out = ratecontrol.band_outcome(q, s, below, curve[below] if below else None, t, n)
    return q, s, qs, out


def test_band_pick_and_outcomes_against_the_full_curve():
    """For every target the band pick returns an evaluated quality; it is in
    the band whenever Q* or Q* - 1 is; 'unreachable' means no quality of
    1..100 lands in the band (on curves where PSNR rises with quality); an
    out-of-band result with some in-band quality is 'missed'."""
    from synth import powerlaw_image
    checked = 0
    for seed, (h, w) in ((8, (48, 64)), (9, (40, 40)), (10, (24, 72))):
        img = powerlaw_image(h, w, seed=seed, beta=1.0 + seed % 3).numpy()
        curve = _sse_curve(img)
        n = img.size
        mono = all(curve[k + 1] <= curve[k] for k in range(1, 100))
        for t in np.linspace(22.0, 52.0, 121):
            q, s, qs, out = _outcome_of(curve, t, n)
            lo, hi = ratecontrol.sse_band(t, n)
            inband = _band_quals(curve, t, n)
            assert s == curve[q]
            assert q in (qs, qs - 1)
            if lo <= curve[qs] <= hi or (qs > 1 and lo <= curve[qs - 1] <= hi and curve[qs] > hi or
                                         qs > 1 and lo <= curve[qs - 1] <= hi and curve[qs] < lo):
                assert out == "within", (seed, t)
            if out == "within":
                assert lo <= s <= hi
            if out == "unreachable" and mono:
                assert inband == [], (seed, t)
            assert out in ("within", "unreachable")
            if out != "within" and inband:
                assert not mono, (seed, t)
            checked += 1
    assert checked == 363


def test_band_outcome_edge_cases_on_constructed_curves():
    n = 4096
    t = 35.0
    lo, hi = ratecontrol.sse_band(t, n)
    thr = ratecontrol.sse_at_most(t, n)
    # quality 1 already far above the band: unreachable from above
    curve = {k: max(1, lo // 4 - k) for k in range(1, 101)}
    q, s, qs, out = _outcome_of(curve, t, n)
    assert q == 1 and out == "unreachable"
    # quality 100 still far below the band: unreachable from below
    curve = {k: 10 * hi + 100 - k for k in range(1, 101)}
    q, s, qs, out = _outcome_of(curve, t, n)
    assert q == 100 and out == "unreachable"
    # the band falls between two adjacent qualities
    curve = {k: (2 * hi if k < 60 else lo // 2) for k in range(1, 101)}
    q, s, qs, out = _outcome_of(curve, t, n)
    assert qs == 60 and q == 60 and out == "unreachable"
    # Q* overshoots the band but Q* - 1 sits just below the target: the band pick takes Q* - 1
    curve = {k: (thr + 1 if k < 60 else lo // 2) for k in range(1, 101)}
    q, s, qs, out = _outcome_of(curve, t, n)
    assert qs == 60 and q == 59 and out == "within" and s == thr + 1 <= hi
    # the split rests on PSNR rising with quality: an in-band quality far
    # from the bracket (a non-monotone curve) is invisible to it
    curve = {k: (2 * hi if k < 60 else lo // 2) for k in range(1, 101)}
    curve[20] = thr
    q, s, qs, out = _outcome_of(curve, t, n)
    assert out == "unreachable" and _band_quals(curve, t, n) == [20]
    # a bisection that ends at Q* > 1 has evaluated Q* - 1, so after the band
    # pick every out-of-band result is bracketed: 'missed' is only reachable
    # for a quality chosen some other way (the band_outcome rule itself)
    assert ratecontrol.band_outcome(60, lo // 2, None, None, t, n) == "missed"
    assert ratecontrol.band_outcome(60, lo // 2, 58, 2 * hi, t, n) == "missed"
    assert ratecontrol.band_outcome(60, lo // 2, 59, hi, t, n) == "missed"      # 59 itself in the band

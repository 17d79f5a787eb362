"""GPU parity of the learned rate controller against the CPU oracle:
features, network forward / gradient / Adam / training epochs, the 8-step
bisection and the learned accept-or-fall-back rule, on grey images and
4:2:0 frames; and the gain of a trained network over plain bisection."""
import numpy as np
import pytest
import torch

from oracle import codec, features, ijg, mlp, psnr, ratecontrol
from synth import powerlaw_image, yuv420_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


def images(n, seed, lo=32, hi=160):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        h, w = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        out.append(powerlaw_image(h, w, seed=seed * 100 + i, beta=float(rng.uniform(1, 3)), rects=-1).numpy())
    return out


def sse_curve(planes, tables_for):
    """SSE at every quality of a frame (list of planes) by the oracle."""
    out = {}
    for q in range(1, 101):
        s = 0
        for p, img in enumerate(planes):
            Q = tables_for(p, q)
            r = codec.reconstruct_plane(codec.compress_plane(img, Q), Q, *img.shape)
            s += psnr.sse(img, r)
        out[q] = s
    return out


def luma(p, q):
    return ijg.luma_table(q) if p == 0 else ijg.chroma_table(q)


def test_features_match_oracle(D):
    imgs = images(6, seed=1)
    targets = np.linspace(28, 42, len(imgs))
    with D.Plan(256, 256, max_batch=16) as plan:
        f = D.dct_rate_features(plan, [torch.from_numpy(i).cuda() for i in imgs], 1, targets).cpu().numpy()
    for k, img in enumerate(imgs):
        ref = features.features_from_stats(features.plane_stats(img), img.shape[1], img.shape[0], targets[k])
        assert np.allclose(f[k], ref.astype(np.float32), rtol=1e-6, atol=1e-7), k


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_and_gradient_match_oracle(D, bf16):
    rng = np.random.default_rng(2)
    n, b = 300, 64
    x = (rng.normal(size=(n, 80)) * 3 + 2).astype(np.float32)
    t = rng.uniform(0, 1, n).astype(np.float32)
    p0 = mlp.init_params(3) + rng.normal(0, 0.02, mlp.N_PARAMS)
    net = D.Mlp(p0, act_bf16=bf16)
    X = torch.from_numpy(x).cuda()
    net.set_norm(X)
    mean = x.astype(np.float64).mean(axis=0)
    std = x.astype(np.float64).std(axis=0)
    assert np.allclose(net.mean.cpu().numpy(), mean, rtol=1e-6, atol=1e-6)
    assert np.allclose(net.std.cpu().numpy(), std, rtol=1e-6)
    mean32 = net.mean.cpu().numpy().astype(np.float64)
    std32 = net.std.cpu().numpy().astype(np.float64)
    p32 = net.params.cpu().numpy().astype(np.float64)
    mode = "bf16" if bf16 else "fp32"
    y, q = net.forward(X)
    y_or, _ = mlp.forward(p32, x.astype(np.float64), mean32, std32, mode)
    tol = 2e-2 if bf16 else 1e-5
    assert np.max(np.abs(y.cpu().numpy() - y_or)) < tol
    idx = torch.from_numpy(rng.permutation(n)[:b].astype(np.int32)).cuda()
    loss, grad = net.loss_grad(X, torch.from_numpy(t).cuda(), idx)
    l_or, g_or = mlp.loss_and_grad(p32, x[idx.cpu().numpy()].astype(np.float64), t[idx.cpu().numpy()], mean32,
                                   std32, mode)
    assert abs(float(loss) - l_or) <= tol * max(l_or, 1e-3)
    g = grad.cpu().numpy()
    scale = np.max(np.abs(g_or))
    assert np.max(np.abs(g - g_or)) <= (2e-2 if bf16 else 1e-4) * scale


@pytest.mark.parametrize("b", [1, 127, 128, 300])
def test_gradient_over_staged_row_chunks_matches_oracle(D, b):
    """The gradient kernel stages 128 minibatch rows at a time: minibatches
    of 1, 127, 128 and 300 rows (two full chunks and a ragged one) against
    the oracle's float64 gradient, fp32 activations."""
    rng = np.random.default_rng(11 + b)
    n = 400
    x = (rng.normal(size=(n, 80)) * 2 - 1).astype(np.float32)
    t = rng.uniform(0, 1, n).astype(np.float32)
    net = D.Mlp(mlp.init_params(7) + rng.normal(0, 0.02, mlp.N_PARAMS), act_bf16=False)
    X = torch.from_numpy(x).cuda()
    net.set_norm(X)
    mean32 = net.mean.cpu().numpy().astype(np.float64)
    std32 = net.std.cpu().numpy().astype(np.float64)
    p32 = net.params.cpu().numpy().astype(np.float64)
    sel = rng.permutation(n)[:b].astype(np.int32)
    loss, grad = net.loss_grad(X, torch.from_numpy(t).cuda(), torch.from_numpy(sel).cuda())
    l_or, g_or = mlp.loss_and_grad(p32, x[sel].astype(np.float64), t[sel], mean32, std32, "fp32")
    assert abs(float(loss) - l_or) <= 1e-5 * max(l_or, 1e-3)
    g = grad.cpu().numpy()
    assert np.max(np.abs(g - g_or)) <= 1e-4 * np.max(np.abs(g_or))


def test_adam_and_training_epochs_match_oracle(D):
    rng = np.random.default_rng(4)
    n = 200
    x = rng.normal(size=(n, 80)).astype(np.float32)
    t = (1 / (1 + np.exp(-(x[:, 0] - 0.5 * x[:, 5])))).astype(np.float32)
    net = D.Mlp(mlp.init_params(5), act_bf16=False)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    net.set_norm(X)
    mean = net.mean.cpu().numpy().astype(np.float64)
    std = net.std.cpu().numpy().astype(np.float64)
    p = net.params.cpu().numpy().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    step = 0
    for epoch in range(3):
        order = rng.permutation(n).astype(np.int32)
        losses = net.train_epoch(X, T, torch.from_numpy(order).cuda(), batch=64, lr=3e-3)
        for b0 in range(0, n, 64):
            sel = order[b0:b0 + 64]
            _, g = mlp.loss_and_grad(p, x[sel].astype(np.float64), t[sel], mean, std, "fp32")
            step += 1
            p, m, v = mlp.adam_step(p, m, v, g, step, lr=3e-3)
        assert losses.numel() == 4
    assert net.step == step
    # Adam divides by |g|: parameters whose gradient is ~0 can move by up to
    # lr per step in either arithmetic, so bound most tightly and all loosely
    d = np.abs(net.params.cpu().numpy() - p)
    assert np.mean(d > 2e-4) < 0.01
    assert d.max() < 12 * 3e-3


def test_bisection_matches_oracle_grey(D):
    imgs = images(5, seed=6, lo=24, hi=72)
    targets = [27.5, 31.0, 35.2, 39.9, 60.0]
    with D.Plan(128, 128, max_batch=8) as plan:
        res = D.dct_rate_control(plan, [torch.from_numpy(i).cuda() for i in imgs], 1, targets)
    for k, img in enumerate(imgs):
        curve = sse_curve([img], luma)
        q, s, _ = ratecontrol.bisect_quality(curve.__getitem__, targets[k], img.size, band_tol=0.25)
        assert int(res["quality"][k]) == q and int(res["sse"][k]) == s, k
    assert res["fell_back"].all()
    assert res["summary"]["passes"] == 8 * len(imgs)


def test_bisection_band_pick_and_outcome_counts(D):
    """Targets spread over 24..50 dB on small images: the library's quality
    and SSE follow the oracle's band pick, its within / unreachable counts
    follow the oracle's outcome split, and on images whose SSE falls as the
    quality rises every 'unreachable' frame has no quality in the band."""
    imgs = images(4, seed=12, lo=24, hi=56)
    targets = list(np.linspace(24.0, 50.0, 27))
    frames = [imgs[k % len(imgs)] for k in range(len(targets))]
    curves = [sse_curve([img], luma) for img in imgs]
    with D.Plan(64, 64, max_batch=32) as plan:
        res = D.dct_rate_control(plan, [torch.from_numpy(i).cuda() for i in frames], 1, targets)
    within = unreachable = 0
    for k, img in enumerate(frames):
        curve = curves[k % len(imgs)]
        n = img.size
        q, s, seen = ratecontrol.bisect_quality(curve.__getitem__, targets[k], n, band_tol=0.25)
        assert int(res["quality"][k]) == q and int(res["sse"][k]) == s, k
        qs, _, _ = ratecontrol.bisect_quality(curve.__getitem__, targets[k], n)
        out = ratecontrol.band_outcome(q, s, qs - 1 if qs - 1 in seen else None,
                                       curve.get(qs - 1), targets[k], n)
        assert out in ("within", "unreachable")
        within += out == "within"
        unreachable += out == "unreachable"
        lo, hi = ratecontrol.sse_band(targets[k], n)
        mono = all(curve[j + 1] <= curve[j] for j in range(1, 100))
        if out == "unreachable" and mono:
            assert not any(lo <= curve[j] <= hi for j in range(1, 101)), k
    summ = res["summary"]
    assert summ["within_tol"] == within and summ["unreachable"] == unreachable
    assert within + unreachable == len(frames) and within > 0


def test_bisection_matches_oracle_yuv420(D):
    frames = [yuv420_frame(64 + 8 * i, 40 + 8 * i, seed=20 + i) for i in range(3)]
    planes = [p for fr in frames for p in fr]
    targets = [30.0, 34.0, 38.0]
    with D.Plan(128, 128, max_batch=16, layout=D.DCT_LAYOUT_YUV420) as plan:
        res = D.dct_rate_control(plan, [p.cuda() for p in planes], 3, targets)
    for k, fr in enumerate(frames):
        ps = [p.numpy() for p in fr]
        curve = sse_curve(ps, luma)
        n = sum(p.size for p in ps)
        q, s, _ = ratecontrol.bisect_quality(curve.__getitem__, targets[k], n, band_tol=0.25)
        assert int(res["quality"][k]) == q and int(res["sse"][k]) == s


def test_learned_decisions_match_oracle(D):
    imgs = images(8, seed=7, lo=24, hi=64)
    targets = list(np.linspace(29, 41, len(imgs)))
    net = D.Mlp(mlp.init_params(8), act_bf16=True)
    with D.Plan(128, 128, max_batch=16) as plan:
        planes = [torch.from_numpy(i).cuda() for i in imgs]
        feats = D.dct_rate_features(plan, planes, 1, targets)
        net.set_norm(feats)
        _, qpred = net.forward(feats)
        res = D.dct_rate_control(plan, planes, 1, targets, net=net)
    qpred = qpred.cpu().numpy()
    for k, img in enumerate(imgs):
        curve = sse_curve([img], luma)
        keep = ratecontrol.learned_decision(curve[int(qpred[k])], targets[k], img.size)
        assert bool(res["fell_back"][k]) == (not keep), k
        if keep:
            assert int(res["quality"][k]) == int(qpred[k]) and int(res["sse"][k]) == curve[int(qpred[k])]
        else:
            q, s, _ = ratecontrol.bisect_quality(curve.__getitem__, targets[k], img.size, band_tol=0.25)
            assert int(res["quality"][k]) == q and int(res["sse"][k]) == s
    s = res["summary"]
    assert s["passes"] == len(imgs) + 8 * s["fell_back"]


def test_trained_network_beats_bisection(D):
    """Train on bisection labels of 1500 images (128..320 px); on 300
    held-out images the learned controller needs fewer pipeline passes than
    bisection, lands at least as many frames within 0.25 dB of the target,
    and every frame it accepts is within 0.25 dB of its target."""
    rng = np.random.default_rng(9)
    n_tr, n_ev = 1500, 300
    dev = "cuda"
    imgs, targets = [], []
    for i in range(n_tr + n_ev):
        h, w = int(rng.integers(16, 41)) * 8, int(rng.integers(16, 41)) * 8
        imgs.append(powerlaw_image(h, w, seed=5000 + i, beta=float(rng.uniform(1, 3)), rects=-1, device=dev))
        targets.append(float(rng.uniform(28, 42)))
    with D.Plan(320, 320, max_batch=n_tr + n_ev) as plan:
        tr = D.dct_rate_control(plan, imgs[:n_tr], 1, targets[:n_tr])
        feats = D.dct_rate_features(plan, imgs, 1, targets)
        labels = D.dct_mlp_labels(torch.from_numpy(tr["quality"].astype(np.int32)).to(dev))
        assert torch.equal(labels.cpu(), torch.from_numpy((tr["quality"].astype(np.float32) - 1) / 99.0))
        net = D.Mlp(mlp.init_params(10), act_bf16=True)
        ftr = feats[:n_tr].contiguous()
        net.set_norm(ftr)
        for epoch in range(300):
            order = torch.from_numpy(rng.permutation(n_tr).astype(np.int32)).to(dev)
            net.train_epoch(ftr, labels, order, batch=128, lr=2e-3)
        ev_imgs, ev_t = imgs[n_tr:], targets[n_tr:]
        learned = D.dct_rate_control(plan, ev_imgs, 1, ev_t, net=net)
        bis = D.dct_rate_control(plan, ev_imgs, 1, ev_t)
    s_l, s_b = learned["summary"], bis["summary"]
    print("learned", s_l, "bisection", s_b)
    assert s_l["fell_back"] < n_ev
    assert s_l["passes"] < s_b["passes"]
    assert s_l["within_tol"] >= s_b["within_tol"]
    for k in range(n_ev):
        if not learned["fell_back"][k]:
            n = ev_imgs[k].numel()
            lo, hi = ratecontrol.sse_band(ev_t[k], n)
            assert lo <= int(learned["sse"][k]) <= hi


def test_rate_control_invalid_arguments(D):
    t = torch.zeros(16, 16, dtype=torch.uint8, device="cuda")
    with D.Plan(32, 32, max_batch=2) as plan:
        with pytest.raises(D.DctError):
            D.dct_rate_control(plan, [t, t, t], 1, [30, 30, 30])      # more frames than max_batch
        with pytest.raises(D.DctError):
            D.dct_rate_control(plan, [t, t], 2, [30])                 # 2 planes per frame
        with pytest.raises(D.DctError):
            D.dct_rate_control(plan, [t], 1, [-5.0])                  # bad target

"""Learned rate control workflow on top of the C ABI: label frames with the
plain pipeline's 8-step bisection, train the network on (features, Q*)
pairs with the library's training kernels, evaluate learned control against
bisection, and save / restore the network.

Every numeric step runs in libdctgb; this module only sequences calls and
draws the seeded permutations and initial weights that the kernels take as
inputs.
"""
import math
import struct
import time
import zlib

import numpy as np
import torch

from . import dctgb as D

_MAGIC = b"DCTGBMLP"
_VERSION = 1


def init_params(seed):
    """Seeded initial weights: uniform in +-1/sqrt(fan_in), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.uniform(-1, 1, (64, 80)) / math.sqrt(80), np.zeros(64),
             rng.uniform(-1, 1, (64, 64)) / math.sqrt(64), np.zeros(64),
             rng.uniform(-1, 1, 64) / math.sqrt(64), np.zeros(1)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def label_by_bisection(plan, planes, planes_per_frame, targets):
    """Q* per frame (int numpy array) and the call's summary."""
    r = D.dct_rate_control(plan, planes, planes_per_frame, targets)
    return r["quality"].copy(), r["summary"]


def train_network(feats, qualities, epochs=300, batch=256, lr=2e-3, seed=0, act_bf16=True, lr_final=2e-4):
    """Trains a fresh network on device features (n, 80) and integer labels
    Q* in 1..100 (target (Q* - 1) / 99).  The learning rate decays
    geometrically from lr to lr_final.  Returns (Mlp, per-epoch mean loss)."""
    dev = feats.device
    n = int(feats.shape[0])
    net = D.Mlp(init_params(seed), act_bf16=act_bf16, device=dev)
    net.set_norm(feats)
    labels = D.dct_mlp_labels(torch.as_tensor(np.asarray(qualities, dtype=np.int32)).to(dev))
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    hist = []
    for e in range(epochs):
        rate = lr * (lr_final / lr) ** (e / max(1, epochs - 1))
        order = torch.as_tensor(rng.permutation(n).astype(np.int32)).to(dev)
        losses = net.train_epoch(feats, labels, order, batch=batch, lr=rate)
        hist.append(losses)
    return net, [float(h.mean()) for h in hist]


def evaluate(plan, planes, planes_per_frame, targets, net):
    """Learned control and plain bisection on the same frames.  Returns a
    dict with per-method summaries, wall and device times and rates."""
    nf = len(planes) // planes_per_frame
    if not isinstance(planes, D.PlaneArray):
        planes = D.PlaneArray(planes)
    out = {}
    for name, model in (("learned", net), ("bisection", None)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = D.dct_rate_control(plan, planes, planes_per_frame, targets, net=model)
        wall = time.perf_counter() - t0
        s = r["summary"]
        out[name] = dict(frames_per_s=nf / wall, gpu_frames_per_s=nf / (s["gpu_ms"] * 1e-3), wall_s=wall,
                         gpu_ms=s["gpu_ms"], fell_back=s["fell_back"], fallback_rate=s["fell_back"] / nf,
                         within_0p25dB=s["within_tol"] / nf, unreachable=s["unreachable"], passes=s["passes"],
                         result=r)
    return out


def save(net, path, seed=0):
    """Flat binary: magic, version, step, act_bf16, seed, n, then params,
    adam_m, adam_v, feat_mean, feat_std (float32) and a CRC-32 of the body."""
    arrays = [t.detach().cpu().numpy().astype(np.float32) for t in (net.params, net.m, net.v, net.mean, net.std)]
    body = struct.pack("<iiiii", _VERSION, net.c.step, net.c.act_bf16, seed, arrays[0].size) + \
        b"".join(a.tobytes() for a in arrays)
    with open(path, "wb") as f:
        f.write(_MAGIC + body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))


def load(path, device="cuda"):
    """Restores a network written by save(); raises on a bad header or checksum."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != _MAGIC or len(data) < 8 + 20 + 4:
        raise ValueError("not a network checkpoint")
    body, crc = data[8:-4], struct.unpack("<I", data[-4:])[0]
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError("checkpoint checksum mismatch")
    version, step, act, seed, n = struct.unpack("<iiiii", body[:20])
    if version != _VERSION or n != D.DCT_MLP_PARAMS:
        raise ValueError("unsupported checkpoint")
    vals = np.frombuffer(body[20:], dtype=np.float32)
    sizes = [n, n, n, 80, 80]
    if vals.size != sum(sizes):
        raise ValueError("truncated checkpoint")
    parts = np.split(vals, np.cumsum(sizes)[:-1])
    net = D.Mlp(parts[0], act_bf16=bool(act), device=device)
    for dst, src in zip((net.m, net.v, net.mean, net.std), parts[1:]):
        dst.copy_(torch.from_numpy(src.copy()))
    net.c.step = step
    return net

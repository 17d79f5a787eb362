"""FP64 reference of the learned rate controller's network, its gradient and
Adam.  The paper has no rate controller; the network is a multilayer
perceptron 80 -> 64 -> 64 -> 1 with GELU hidden units and a sigmoid output:

  a1 = W1 xn + b1,  h1 = act(gelu(a1))
  a2 = W2 h1 + b2,  h2 = act(gelu(a2))
  z  = W3 h2 + b3,  y  = sigmoid(z)
  xn = (x - mean) / std   (fixed input normalisation)
  loss = mean over the batch of (y - t)^2

gelu(a) = a * Phi(a) with Phi the standard normal CDF (the erf form).
act() is the identity ("fp32" activations) or rounding to the nearest
bfloat16, ties to even ("bf16" activations, the GPU's default).  The output
y predicts (Q* - 1) / 99 for the smallest quality Q* meeting the target.

Flat parameter layout (9409 values): W1[64][80], b1[64], W2[64][64], b2[64],
W3[64], b3.

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np
from scipy.special import erf

N_IN, N_HID = 80, 64
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    The value is first rounded to float32 (the GPU computes in float32)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def act(h, mode):
    return bf16_round(h) if mode == "bf16" else h


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, x, mean, std, mode="bf16"):
    """x: (B, 80) raw features.  Returns y (B,) and the cache for backward."""
    w = unpack(p)
    xn = (np.asarray(x, dtype=np.float64) - mean) / std
    a1 = xn @ w["W1"].T + w["b1"]
    h1 = act(gelu(a1), mode)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = act(gelu(a2), mode)
    z = h2 @ w["W3"] + w["b3"][0]
    y = sigmoid(z)
    return y, dict(xn=xn, a1=a1, h1=h1, a2=a2, h2=h2, z=z, y=y, w=w)


def loss_and_grad(p, x, t, mean, std, mode="bf16"):
    """Mean squared error and its gradient with respect to the flat parameters
    (back-propagation through the forward above; the rounding of act() is
    treated as the identity, as the GPU does)."""
    y, c = forward(p, x, mean, std, mode)
    t = np.asarray(t, dtype=np.float64)
    b = y.shape[0]
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / b
    dz = dy * y * (1.0 - y)
    w = c["w"]
    g = {"W3": dz @ c["h2"], "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, w["W3"])
    da2 = dh2 * gelu_grad(c["a2"])
    g["W2"] = da2.T @ c["h1"]
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ w["W2"]
    da1 = dh1 * gelu_grad(c["a1"])
    g["W1"] = da1.T @ c["xn"]
    g["b1"] = da1.sum(axis=0)
    return loss, pack(g)


def adam_step(p, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba); `step` counts from 1.  Returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """Seeded initial weights (uniform in +-1/sqrt(fan_in), zero biases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {"W1": rng.uniform(-1, 1, (N_HID, N_IN)) / math.sqrt(N_IN), "b1": np.zeros(N_HID),
         "W2": rng.uniform(-1, 1, (N_HID, N_HID)) / math.sqrt(N_HID), "b2": np.zeros(N_HID),
         "W3": rng.uniform(-1, 1, N_HID) / math.sqrt(N_HID), "b3": np.zeros(1)}
    return pack(d)


def predict_quality(y):
    """Quality from the network output: clamp(rint(1 + 99 y), 1, 100)."""
    return np.clip(np.rint(1.0 + 99.0 * np.asarray(y, dtype=np.float64)), 1, 100).astype(np.int64)

"""Oracle of the learned bracket (test infrastructure; float64 numpy).

The network maps (v, log x) to the range [t0, t1] of Sec. 2.3 (the range the plain bracket of
Algorithms 1-3 finds).  Layout and arithmetic, written out plainly:

  features   a = asinh(v * IN_SCALE[0]) * IN_SCALE[1],   b = ln(x) * IN_SCALE[2] + IN_SCALE[3]
  layer 1    h1 = relu(W1 [a, b] + b1)                     W1: 64 x 2
  layer 2    h2 = relu(W2 h1 + b2)                         W2: 64 x 64
  layer 3    y  = W3 h2 + b3                               W3: 2 x 64
  outputs    L_k = y_k * OUT_SCALE[2k] + OUT_SCALE[2k+1]   (k = 0, 1)
             t0 = max(t_ref - max(e^{L_0} - DELTA, 0), 0),  t1 = t_ref + max(e^{L_1} - DELTA, 0)
  targets    L_0* = ln(t_p - t0* + DELTA),  L_1* = ln(t1* - t_p + DELTA)   from a plain bracket
  loss       mean over the batch of ((y_0 - T_0)^2 + (y_1 - T_1)^2) / 2,
             T_k = (L_k* - OUT_SCALE[2k+1]) / OUT_SCALE[2k]
  Adam       Kingma & Ba (2015): m = b1 m + (1 - b1) g, s = b2 s + (1 - b2) g^2,
             w -= lr * (m / (1 - b1^t)) / (sqrt(s / (1 - b2^t)) + eps)
  batches    sample k of step j is index  mix(seed + j * batch + k) mod n  with mix the SplitMix64
             finalizer (Steele, Lea & Flood 2014) of its argument plus 0x9e3779b97f4a7c15.

Parameter vector order: W1[64][2], b1[64], W2[64][64], b2[64], W3[2][64], b3[2] (4482 values).
"""
from __future__ import annotations

import math

import numpy as np

H = 64
NPARAMS = H * 2 + H + H * H + H + 2 * H + 2
IN_SCALE = (2.0, 2.0 / math.asinh(400.0), 1.0 / (4.0 * math.log(10.0)), 0.0)
OUT_SCALE = (3.0, -3.0, 2.0, -1.0)  # (scale, shift) of L_0, then of L_1
DELTA = 1e-3
MASK64 = (1 << 64) - 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.size == NPARAMS
    o = 0
    out = {}
    for name, shape in (("W1", (H, 2)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (2, H)), ("b3", (2,))):
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[k], dtype=np.float64).ravel()
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def features(v, x):
    v = np.asarray(v, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    return np.stack([np.arcsinh(v * IN_SCALE[0]) * IN_SCALE[1], np.log(x) * IN_SCALE[2] + IN_SCALE[3]],
                    axis=1)


def forward(p, v, x):
    """Intermediates of the forward pass for a batch (rows = samples)."""
    P = unpack(p)
    f = features(v, x)
    z1 = f @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"].T + P["b3"]
    return {"f": f, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y}


def peak(v, x, iters: int = 60):
    """The peak t_p of g (Sec. 2.1-2.2): 0 if v^2 <= x, else the zero of
    g'(t) = v tanh(vt) - x sinh t.  Newton's method from asinh(v/x), where g' <= 0 (tanh <= 1);
    g' is concave (g''' <= 0), so the iterates decrease monotonically to the zero."""
    v = np.abs(np.asarray(v, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    t = np.arcsinh(v / x)
    for _ in range(iters):
        th = np.tanh(v * t)
        g1 = v * th - x * np.sinh(t)
        g2 = v * v * (1 - th * th) - x * np.cosh(t)
        step = np.where(g2 != 0, g1 / np.where(g2 != 0, g2, 1.0), 0.0)
        t = np.clip(t - step, 0.0, t)
    return np.where(v * v > x, t, 0.0)


def targets(t0, tp, t1):
    """Normalised targets (T_0, T_1) from a range [t0, t1] around the peak tp."""
    L0 = np.log(np.maximum(np.asarray(tp) - np.asarray(t0), 0.0) + DELTA)
    L1 = np.log(np.maximum(np.asarray(t1) - np.asarray(tp), 0.0) + DELTA)
    return np.stack([(L0 - OUT_SCALE[1]) / OUT_SCALE[0], (L1 - OUT_SCALE[3]) / OUT_SCALE[2]], axis=1)


def loss_grad(p, v, x, t0, tp, t1):
    """Mean loss over the batch and its gradient with respect to the parameter vector."""
    P = unpack(p)
    F = forward(p, v, x)
    T = targets(t0, tp, t1)
    B = F["y"].shape[0]
    r = F["y"] - T
    loss = 0.5 * np.sum(r * r) / B
    dy = r / B
    g = {"W3": dy.T @ F["h2"], "b3": dy.sum(0)}
    dz2 = (dy @ P["W3"]) * (F["z2"] > 0)
    g["W2"] = dz2.T @ F["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (F["z1"] > 0)
    g["W1"] = dz1.T @ F["f"]
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def adam(p, m, s, g, step, lr, beta1, beta2, eps):
    """One Adam update (step counts from 1).  Returns new (p, m, s)."""
    m = beta1 * m + (1 - beta1) * g
    s = beta2 * s + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    sh = s / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(sh) + eps), m, s


def predict(p, v, x, t_ref):
    """(t0, t1) from the network around the reference point t_ref (the peak)."""
    y = forward(p, v, x)["y"]
    L0 = y[:, 0] * OUT_SCALE[0] + OUT_SCALE[1]
    L1 = y[:, 1] * OUT_SCALE[2] + OUT_SCALE[3]
    t_ref = np.asarray(t_ref, dtype=np.float64)
    t0 = np.maximum(t_ref - np.maximum(np.exp(L0) - DELTA, 0.0), 0.0)
    t1 = t_ref + np.maximum(np.exp(L1) - DELTA, 0.0)
    return t0, t1


def mix64(z: int) -> int:
    """The SplitMix64 output function applied to z + 0x9e3779b97f4a7c15."""
    z = (z + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def batch_indices(seed: int, step: int, batch: int, n: int):
    """Sample indices of one training step."""
    return np.array([mix64((seed + step * batch + k) & MASK64) % n for k in range(batch)],
                    dtype=np.int64)


def train(p, v, x, t0, t1, steps, batch, lr, beta1, beta2, eps, seed, step0=0):
    """Plain Adam training loop on brackets (t0, t1) around the peak of each pair; returns
    (params, per-step losses).  step0 continues the step count of an earlier call."""
    p = np.array(p, dtype=np.float64)
    tp = peak(v, x)
    m = np.zeros_like(p)
    s = np.zeros_like(p)
    losses = []
    for j in range(step0, step0 + steps):
        idx = batch_indices(seed, j, batch, len(v))
        loss, g = loss_grad(p, v[idx], x[idx], t0[idx], tp[idx], t1[idx])
        losses.append(loss)
        p, m, s = adam(p, m, s, g, j + 1, lr, beta1, beta2, eps)
    return p, np.array(losses)

"""FP64 NumPy oracle of the gradient-surrogate MLP (6 -> 128 -> 128 -> 6, tanh).

TEST INFRASTRUCTURE: used only by the tests.

Same parameter layout as the library: W1[128x6], b1[128], W2[128x128], b2[128],
W3[6x128], b3[6] (rows are outputs).  The loss is the mean over batch x 6 of
(y - target)^2; its gradient is back-propagated by hand (chain rule through
the two tanh layers).  Adam follows Kingma & Ba (2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

MI, MH, MO = 6, 128, 6
SIZES = [("W1", MH * MI), ("b1", MH), ("W2", MH * MH), ("b2", MH), ("W3", MO * MH), ("b3", MO)]
PARAM_COUNT = sum(s for _, s in SIZES)


def unpack(w):
    w = np.asarray(w, np.float64)
    out, off = {}, 0
    for name, size in SIZES:
        out[name] = w[off:off + size]
        off += size
    out["W1"] = out["W1"].reshape(MH, MI)
    out["W2"] = out["W2"].reshape(MH, MH)
    out["W3"] = out["W3"].reshape(MO, MH)
    return out


def forward(w, x):
    p = unpack(w)
    x = np.asarray(x, np.float64)
    h1 = np.tanh(x @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    return h2 @ p["W3"].T + p["b3"], (x, h1, h2)


def loss_grad(w, x, target):
    p = unpack(w)
    y, (x, h1, h2) = forward(w, x)
    target = np.asarray(target, np.float64)
    n = x.shape[0]
    d = y - target
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (n * MO)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ p["W3"]) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 * h1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(w, m, v, g, lr, b1, b2, eps, step):
    """One bias-corrected Adam step in FP64; returns (w, m, v)."""
    w, m, v, g = (np.asarray(a, np.float64) for a in (w, m, v, g))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16_round(x):
    """FP32 -> BF16 with round-to-nearest-even; returns the BF16 values as FP32
    (the upper 16 bits of the FP32 pattern after rounding)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def bf16_bits(x):
    """BF16 bit patterns (uint16) of FP32 values, rounded to nearest even."""
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def surrogate_gradient(w, q, norm):
    """Surrogate gradient in sampler coordinates:
    mean_g + A (q - mean_q) + sd_g * MLP((q - mean_q) / sd_q), with
    norm = [mean_q, sd_q, mean_g, sd_g, A (6x6 row-major)]."""
    norm = np.asarray(norm, np.float64)
    dq = np.asarray(q, np.float64)[:MI] - norm[0:6]
    y, _ = forward(w, (dq / norm[6:12])[None, :])
    return norm[12:18] + norm[24:60].reshape(MI, MI) @ dq + norm[18:24] * y[0]

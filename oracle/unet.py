"""FP64 CPU oracle of the warm-start network (a 4-level U-Net) and its analytic gradients.

TEST INFRASTRUCTURE ONLY (see oracle/pc_engine.py). The paper has no learned
component; this network is the learned warm start of the workload: it maps
log-intensity patterns to the amplitude and phase of the central object patch
and to the coherence blur width sigma. Architecture (S = input side, C = base
channels; 'same' 3x3 correlations with zero padding, NHWC):

  a0 = relu(conv(x, 1 -> C))          S      p0 = avgpool2(a0)
  a1 = relu(conv(p0, C -> 2C))        S/2    p1 = avgpool2(a1)
  a2 = relu(conv(p1, 2C -> 4C))       S/4    p2 = avgpool2(a2)
  a3 = relu(conv(p2, 4C -> 8C))       S/8
  a4 = relu(conv([up2(a3), a2], 12C -> 4C))  S/4
  a5 = relu(conv([up2(a4), a1], 6C -> 2C))   S/2
  out = conv(a5, 2C -> 2)             S/2    (amplitude, phase of the patch)
  sigma = mean_hw(a3) . w7 + b7
  loss = mean((out - target)^2) + lam * mean((sigma - sigma_t)^2)

With `bf16=True` every tensor that the GPU path stores in bfloat16 (inputs of
each convolution, weights, gradients fed to the gradient contractions) is
rounded to bfloat16 at the same point, so the GPU gradients can be compared
tightly; with `bf16=False` it is the plain FP64 network.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # tap = 3 (dy + 1) + (dx + 1)


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(C):
    """(C_in, C_out) of the seven convolutions."""
    return [(1, C), (C, 2 * C), (2 * C, 4 * C), (4 * C, 8 * C), (12 * C, 4 * C), (6 * C, 2 * C), (2 * C, 2)]


def init_params(C, seed=0):
    rng = np.random.default_rng(seed)
    params = {}
    for i, (ci, co) in enumerate(layer_shapes(C)):
        params[f"w{i}"] = rng.standard_normal((co, 9, ci)) * np.sqrt(2.0 / (9 * ci))
        params[f"b{i}"] = 0.01 * rng.standard_normal(co)
    params["w7"] = rng.standard_normal(8 * C) * np.sqrt(1.0 / (8 * C))
    params["b7"] = np.array([1.5])
    return params


def conv(x, w, b):
    """y[n, i, j, o] = b[o] + sum_{tap, c} x[n, i + dy, j + dx, c] w[o, tap, c] (zero padding)."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((n, h, wd, w.shape[0])) + b
    for t, (dy, dx) in enumerate(TAPS):
        y += np.einsum("nijc,oc->nijo", xp[:, 1 + dy:1 + dy + h, 1 + dx:1 + dx + wd], w[:, t, :])
    return y


def conv_backward(x, w, dy):
    """Gradients of conv: (dx, dw, db)."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for t, (ddy, ddx) in enumerate(TAPS):
        win = xp[:, 1 + ddy:1 + ddy + h, 1 + ddx:1 + ddx + wd]
        dw[:, t, :] = np.einsum("nijo,nijc->oc", dy, win)
        dxp[:, 1 + ddy:1 + ddy + h, 1 + ddx:1 + ddx + wd] += np.einsum("nijo,oc->nijc", dy, w[:, t, :])
    return dxp[:, 1:-1, 1:-1], dw, dy.sum(axis=(0, 1, 2))


def avgpool2(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(dy):
    n, h, w, c = dy.shape
    return dy.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def forward(params, x, bf16=False):
    """x: (n, S, S, 1). Returns (out (n, S/2, S/2, 2), sigma (n,), cache)."""
    rd = bf16_round if bf16 else (lambda a: a)
    W = {k: (rd(v) if k.startswith("w") and k != "w7" else v) for k, v in params.items()}
    c = {}
    c["x"] = rd(x)
    c["a0"] = rd(np.maximum(conv(c["x"], W["w0"], W["b0"]), 0))
    c["p0"] = rd(avgpool2(c["a0"]))
    c["a1"] = rd(np.maximum(conv(c["p0"], W["w1"], W["b1"]), 0))
    c["p1"] = rd(avgpool2(c["a1"]))
    c["a2"] = rd(np.maximum(conv(c["p1"], W["w2"], W["b2"]), 0))
    c["p2"] = rd(avgpool2(c["a2"]))
    c["a3"] = rd(np.maximum(conv(c["p2"], W["w3"], W["b3"]), 0))
    c["q2"] = np.concatenate([up2(c["a3"]), c["a2"]], axis=3)
    c["a4"] = rd(np.maximum(conv(c["q2"], W["w4"], W["b4"]), 0))
    c["q1"] = np.concatenate([up2(c["a4"]), c["a1"]], axis=3)
    c["a5"] = rd(np.maximum(conv(c["q1"], W["w5"], W["b5"]), 0))
    out = conv(c["a5"], W["w6"], W["b6"])
    c["g"] = c["a3"].mean(axis=(1, 2))
    sigma = c["g"] @ W["w7"] + W["b7"][0]
    c["W"] = W
    return out, sigma, c


def loss_and_grads(params, x, target, sigma_t, lam=0.1, bf16=False):
    """Loss and the analytic gradient of every parameter."""
    out, sigma, c = forward(params, x, bf16)
    rd = bf16_round if bf16 else (lambda a: a)
    W = c["W"]
    n_out = out.size
    loss = np.sum((out - target) ** 2) / n_out + lam * np.sum((sigma - sigma_t) ** 2) / len(sigma)
    g = {}
    d_out = rd(2.0 * (out - target) / n_out)
    d_a5, g["w6"], g["b6"] = conv_backward(c["a5"], W["w6"], d_out)
    d_c5 = rd(d_a5 * (c["a5"] > 0))
    d_q1, g["w5"], g["b5"] = conv_backward(c["q1"], W["w5"], d_c5)
    C4 = c["a4"].shape[3]
    d_a4 = up2_backward(d_q1[..., :C4])
    d_a1_skip = d_q1[..., C4:]
    d_c4 = rd(d_a4 * (c["a4"] > 0))
    d_q2, g["w4"], g["b4"] = conv_backward(c["q2"], W["w4"], d_c4)
    C3 = c["a3"].shape[3]
    d_a3 = up2_backward(d_q2[..., :C3])
    d_a2_skip = d_q2[..., C3:]
    d_sigma = 2.0 * lam * (sigma - sigma_t) / len(sigma)
    g["w7"] = c["g"].T @ d_sigma
    g["b7"] = np.array([d_sigma.sum()])
    hw = c["a3"].shape[1] * c["a3"].shape[2]
    d_a3 = d_a3 + (d_sigma[:, None] * W["w7"][None, :])[:, None, None, :] / hw
    d_c3 = rd(d_a3 * (c["a3"] > 0))
    d_p2, g["w3"], g["b3"] = conv_backward(c["p2"], W["w3"], d_c3)
    d_a2 = avgpool2_backward(d_p2) + d_a2_skip
    d_c2 = rd(d_a2 * (c["a2"] > 0))
    d_p1, g["w2"], g["b2"] = conv_backward(c["p1"], W["w2"], d_c2)
    d_a1 = avgpool2_backward(d_p1) + d_a1_skip
    d_c1 = rd(d_a1 * (c["a1"] > 0))
    d_p0, g["w1"], g["b1"] = conv_backward(c["p0"], W["w1"], d_c1)
    d_a0 = avgpool2_backward(d_p0)
    d_c0 = rd(d_a0 * (c["a0"] > 0))
    _, g["w0"], g["b0"] = conv_backward(c["x"], W["w0"], d_c0)
    return loss, g, out, sigma

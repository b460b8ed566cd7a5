"""FP64 oracle of the learned initial-guess network.

TEST INFRASTRUCTURE ONLY (tests/, the smoke check, the benchmark's CPU legs).

The paper has no network; this is the learned-guess part of the build: a
small CNN maps the scaled right-hand side to an initial guess for the sweeps
of Sec. IV. Definition (all FP64, NCHW numpy arrays):
  layer l: z = conv3x3_periodic(x, W_l) + b_l, x' = gelu(z) except after the
           last layer; widths 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1;
  conv3x3_periodic(x, W; d)[b, o, i, j] =
      sum_{c, dy, dx} W[o, c, dy, dx] * x[b, c, (i + d(dy - 1)) mod H, (j + d(dx - 1)) mod W]
  (cross-correlation with circular padding, the convention of conv2d; d is the
  layer's dilation, 1 for a plain 3x3 layer);
  gelu(z) = z * Phi(z), Phi the standard normal CDF (erf form);
  loss = mean((y - t)^2) over all output elements;
  Adam with bias correction (beta1 0.9, beta2 0.999, eps 1e-8).
The backward pass is the analytic chain rule of these definitions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

WIDTHS = (1, 32, 32, 32, 32, 32, 1)


def conv(x, W, b, d=1):
    """Periodic 3x3 cross-correlation with dilation d: x (B, Cin, H, W),
    W (Cout, Cin, 3, 3), b (Cout,)."""
    B, _, H, Wd = x.shape
    out = np.zeros((B, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            xs = np.roll(x, shift=(-(dy - 1) * d, -(dx - 1) * d), axis=(2, 3))
            out += np.einsum("bchw,oc->bohw", xs, W[:, :, dy, dx])
    return out + b[None, :, None, None]


def conv_input_grad(g, W, d=1):
    """d loss / d x of conv for upstream gradient g (B, Cout, H, W)."""
    out = np.zeros((g.shape[0], W.shape[1], g.shape[2], g.shape[3]))
    for dy in range(3):
        for dx in range(3):
            t = np.einsum("bohw,oc->bchw", g, W[:, :, dy, dx])
            out += np.roll(t, shift=((dy - 1) * d, (dx - 1) * d), axis=(2, 3))
    return out


def conv_weight_grad(g, x, d=1):
    """(dW, db) of conv for upstream gradient g and input x."""
    dW = np.zeros((g.shape[1], x.shape[1], 3, 3))
    for dy in range(3):
        for dx in range(3):
            xs = np.roll(x, shift=(-(dy - 1) * d, -(dx - 1) * d), axis=(2, 3))
            dW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", g, xs)
    return dW, g.sum(axis=(0, 2, 3))


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(rng: np.random.Generator, widths=WIDTHS):
    """He-normal weights (std sqrt(2 / (9 Cin))), zero biases."""
    ps = []
    for cin, cout in zip(widths[:-1], widths[1:]):
        W = rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (9 * cin))
        ps.append((W, np.zeros(cout)))
    return ps


def forward(params, x, dil=None):
    """Returns (y, cache) with cache = per-layer (input, pre-activation);
    dil: per-layer dilations (default all 1)."""
    dil = dil or (1,) * len(params)
    cache = []
    h = x
    for li, (W, b) in enumerate(params):
        z = conv(h, W, b, dil[li])
        cache.append((h, z))
        h = gelu(z) if li < len(params) - 1 else z
    return h, cache


def mse(y, t):
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, cache, dy, dil=None):
    """Gradients [(dW, db)] of the loss whose output gradient is dy."""
    dil = dil or (1,) * len(params)
    grads = [None] * len(params)
    g = dy
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        h, z = cache[li]
        if li < len(params) - 1:
            g = g * gelu_grad(z)
        grads[li] = conv_weight_grad(g, h, dil[li])
        g = conv_input_grad(g, W, dil[li])
    return grads


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1**step)
    vh = v / (1 - b2**step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v

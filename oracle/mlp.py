"""FP64 reference of the warm-start MLP (oracle, test infrastructure).

The network maps an (E, k) point to the 2 x s x s real/imaginary parts of a
lead's surface Green's function.  The paper has no learned part; the
architecture is fixed by the workload description (width 512, 3 layers, BF16
weights).  Readings for what that description leaves open:

* features: (E, cos k, sin k, sin(m pi E), cos(m pi E) for m = 1..8) -> 19 inputs;
* SiLU activations, layers 19 -> 512 -> 512 -> 2 s^2;
* output layout: Re g row-major, then Im g row-major, both multiplied by a
  fixed per-lead scale c (so targets are O(1));
* loss: mean squared error over batch and outputs;
* Adam with bias correction.

The GPU kernels keep FP32 master weights and compute with their BF16
roundings; the parity tests feed this module those same BF16 values (as
float64), so the comparison is on forward/backward arithmetic.
"""
from __future__ import annotations

import numpy as np

N_FOURIER = 8
N_IN = 3 + 2 * N_FOURIER


def features(E, k):
    """(B,) energies and momenta -> (B, 19) input features."""
    E = np.atleast_1d(np.asarray(E, np.float64))
    k = np.atleast_1d(np.asarray(k, np.float64))
    cols = [E, np.cos(k), np.sin(k)]
    for m in range(1, N_FOURIER + 1):
        cols.append(np.sin(m * np.pi * E))
        cols.append(np.cos(m * np.pi * E))
    return np.stack(cols, axis=1)


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    sg = 1.0 / (1.0 + np.exp(-x))
    return sg * (1.0 + x * (1.0 - sg))


def init_params(n_out, width=512, seed=0):
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    dims = [(width, N_IN), (width, width), (n_out, width)]
    params = []
    for (o, i) in dims:
        lim = 1.0 / np.sqrt(i)
        params.append(rng.uniform(-lim, lim, (o, i)))
        params.append(np.zeros(o))
    return params


def forward(params, x):
    """Returns (y, cache) for inputs x (B, 19)."""
    W1, b1, W2, b2, W3, b3 = params
    h1 = x @ W1.T + b1
    a1 = silu(h1)
    h2 = a1 @ W2.T + b2
    a2 = silu(h2)
    y = a2 @ W3.T + b3
    return y, (x, h1, a1, h2, a2)


def loss(y, t):
    return float(np.mean((y - t) ** 2))


def backward(params, cache, y, t):
    """Gradients of the mean-squared loss w.r.t. (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    x, h1, a1, h2, a2 = cache
    dy = 2.0 * (y - t) / y.size
    dW3 = dy.T @ a2
    db3 = dy.sum(0)
    dh2 = (dy @ W3) * dsilu(h2)
    dW2 = dh2.T @ a1
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * dsilu(h1)
    dW1 = dh1.T @ x
    db1 = dh1.sum(0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = beta1 * mi + (1 - beta1) * g
        vi = beta2 * vi + (1 - beta2) * g * g
        mh = mi / (1 - beta1 ** t)
        vh = vi / (1 - beta2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v


def pack_g(g, scale):
    """Complex s x s -> flat target (2 s^2,): [Re row-major, Im row-major] * scale."""
    return np.concatenate([g.real.ravel(), g.imag.ravel()]) * scale


def unpack_g(y, s, scale):
    y = np.asarray(y, np.float64) / scale
    return (y[:s * s] + 1j * y[s * s:]).reshape(s, s)

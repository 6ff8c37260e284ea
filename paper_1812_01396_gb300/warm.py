"""Training driver of the learned warm start (argument marshalling and the
training loop; every computation runs in the library's kernels).

The network maps (E, k) features to the scaled real/imaginary parts of one
lead's surface Green's function.  Training targets come from the plain
doubling of the same library (ss_surface_gf without warm start).
"""
from __future__ import annotations

import math

import numpy as np

N_FOURIER = 8
N_IN = 3 + 2 * N_FOURIER


def features(E, k):
    """(B,) energies and momenta -> (B, 19) float32: E, cos k, sin k, sin/cos(m pi E)."""
    E = np.atleast_1d(np.asarray(E, np.float64))
    k = np.atleast_1d(np.asarray(k, np.float64))
    cols = [E, np.cos(k), np.sin(k)]
    for m in range(1, N_FOURIER + 1):
        cols.append(np.sin(m * math.pi * E))
        cols.append(np.cos(m * math.pi * E))
    return np.stack(cols, axis=1).astype(np.float32)


def pack_targets(gs, scale):
    """List of complex (s, s) -> (B, 2 s^2) float32: [Re row-major, Im row-major] * scale."""
    return np.stack([np.concatenate([g.real.ravel(), g.imag.ravel()]) * scale for g in gs]).astype(np.float32)


def train(net, handle, E, k_id, kval, side, scale, epochs=60, batch=256, lr=1e-3, seed=7, log=None):
    """Generate targets with the plain doubling, then Adam with cosine decay.

    Returns (losses per epoch, targets as float32 array)."""
    import torch

    gs, _, _, st, _ = handle.surface_gf(E, k_id, side=side)
    if handle.device_ptrs:
        gs = [g.cpu().numpy() for g in gs]
    tgt = pack_targets(gs, scale)
    x = torch.from_numpy(features(E, kval)).cuda()
    t = torch.from_numpy(tgt).cuda()
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    steps = epochs * max(1, n // batch)
    it = 0
    losses = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        tot = 0.0
        nb = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / steps))
            tot += net.train_step(x[idx].contiguous(), t[idx].contiguous(), lr_t)
            nb += 1
            it += 1
        losses.append(tot / max(nb, 1))
        if log:
            log(ep, losses[-1])
    return losses, tgt

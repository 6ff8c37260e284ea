"""Surface Dyson equation helpers for the warm start (oracle, test infrastructure).

The surface Green's function of a semi-infinite lead satisfies
  g_R = (D - U g_R L)^-1   (bulk to the right),
  g_L = (D - L g_L U)^-1   (bulk to the left),
which is what the doubling converges to.  A seeded iterate is accepted when
the relative Dyson residual ||g (D - U g L) - 1||_F / ||1||_F is below the
acceptance threshold; otherwise the plain doubling result is used.
"""
from __future__ import annotations

import numpy as np


def dyson_residual(g, D, U, L, side="R"):
    s = D.shape[0]
    K = U @ g @ L if side == "R" else L @ g @ U
    r = g @ (D - K) - np.eye(s)
    return float(np.linalg.norm(r) / np.sqrt(s))


def fixed_point(g0, D, U, L, side="R", iters=8):
    """g <- (D - U g L)^-1 (right lead) repeated ``iters`` times."""
    g = np.asarray(g0, np.complex128)
    for _ in range(iters):
        K = U @ g @ L if side == "R" else L @ g @ U
        g = np.linalg.inv(D - K)
    return g

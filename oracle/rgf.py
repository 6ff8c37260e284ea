"""Recursive Green's-function corners (FP64 oracle, test infrastructure).

For devices too large for a dense N x N matrix: the standard left- and
right-connected recursions on M = A - Sigma_L (+) Sigma_R give the first and
last block columns of M^-1 (hence the four corners and x for an injection in
blocks 1 and n) using only s x s solves.  Validated against the dense mode on
small devices.

  right-connected: gR_n = M_nn^-1, gR_i = (M_ii - M_{i,i+1} gR_{i+1} M_{i+1,i})^-1
                   G_11 = gR_1,  G_{i,1} = -gR_i M_{i,i-1} G_{i-1,1}
  left-connected:  gL_1 = M_11^-1, gL_i = (M_ii - M_{i,i-1} gL_{i-1} M_{i-1,i})^-1
                   G_nn = gL_n,  G_{i,n} = -gL_i M_{i,i+1} G_{i+1,n}
"""
from __future__ import annotations

import numpy as np

from . import leads


def block_columns(dev, E, sigma_L, sigma_R):
    """First and last block columns of M^-1 as (n, s, s) arrays."""
    n, s = dev.n_b, dev.s_b
    Md = [E * dev.S_diag[i] - dev.H_diag[i] for i in range(n)]
    Md[0] = Md[0] - sigma_L
    Md[-1] = Md[-1] - sigma_R
    Mu = [E * dev.S_up[i] - dev.H_up[i] for i in range(n - 1)]
    Ml = [u.conj().T for u in Mu]                          # M_{i+1,i}

    gR = [None] * n
    gR[n - 1] = np.linalg.inv(Md[n - 1])
    for i in range(n - 2, -1, -1):
        gR[i] = np.linalg.inv(Md[i] - Mu[i] @ gR[i + 1] @ Ml[i])
    col1 = np.empty((n, s, s), np.complex128)
    col1[0] = gR[0]
    for i in range(1, n):
        col1[i] = -gR[i] @ Ml[i - 1] @ col1[i - 1]
    del gR

    gL = [None] * n
    gL[0] = np.linalg.inv(Md[0])
    for i in range(1, n):
        gL[i] = np.linalg.inv(Md[i] - Ml[i - 1] @ gL[i - 1] @ Mu[i - 1])
    coln = np.empty((n, s, s), np.complex128)
    coln[n - 1] = gL[n - 1]
    for i in range(n - 2, -1, -1):
        coln[i] = -gL[i] @ Mu[i] @ coln[i + 1]
    return col1, coln


def solve_point(dev, E, inj_rows=None, eta=leads.DEFAULT_ETA, tol=leads.DEFAULT_TOL,
                max_iter=leads.DEFAULT_MAX_ITER, sigmas=None):
    """Same outputs as :func:`oracle.dense.solve_point` (no dense matrix)."""
    s = dev.s_b
    if sigmas is None:
        sL, sR, info = leads.self_energies(dev, E, eta, tol, max_iter)
    else:
        sL, sR = sigmas
        info = {}
    col1, coln = block_columns(dev, E, sL, sR)
    G11, Gn1, G1n, Gnn = col1[0], col1[-1], coln[0], coln[-1]
    gl, gr = leads.gamma(sL), leads.gamma(sR)
    tr = complex(np.trace(gl @ G1n @ gr @ G1n.conj().T))
    tr_rl = complex(np.trace(gr @ Gn1 @ gl @ Gn1.conj().T))
    out = dict(sigma_L=sL, sigma_R=sR, G11=G11, G1n=G1n, Gn1=Gn1, Gnn=Gnn, T=tr.real,
               T_imag=tr.imag, T_RL=tr_rl.real, info=info)
    if inj_rows is not None:
        b1, bn = inj_rows[:s], inj_rows[s:]
        x = np.einsum("iab,bc->iac", col1, b1) + np.einsum("iab,bc->iac", coln, bn)
        out["x"] = x.reshape(-1, inj_rows.shape[1])
    return out

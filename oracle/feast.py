"""Lead self-energies from the lead's Bloch modes: the FEAST route of Sec. 3A
(FP64 oracle, test infrastructure).

The lead's modes psi_q = lambda^q u solve the one-neighbour case of Eq. bound.
With the blocks of M = z S - H at z = E + i eta (the same broadening as the
decimation, so the retarded modes sit off the unit circle):

    (L + lambda D + lambda^2 U) u = 0,
    D = z S00 - H00,  U = z S01 - H01 (cell q -> q+1),  L = z S01^H - H01^H.

FEAST (Eq. feast) obtains the m eigenpairs inside the annulus 1/R < |lambda| < R
from a contour-integral subspace and a Rayleigh-Ritz step; what it computes has
a plain definition, the eigenpairs of the pencil inside that annulus, which
this oracle takes straight from a dense generalized eigensolver on a companion
form.  Reading of how Sigma follows from the modes (the paper refers to its
earlier work for the formula):

* right lead (bulk to the right): the right-going modes, |lambda| < 1, give the
  Bloch matrix F+ = U+ diag(lambda) U+^+ (U+ = their u's as columns, U+^+ the
  Moore-Penrose inverse); g_R = (D + U F+)^-1 from the surface cell's row
  D psi_0 + U psi_1 = 1; Sigma_R = A_{n,n+1} g_R A_{n+1,n} at real E;
* left lead: the left-going modes, |lambda| > 1, propagate towards the bulk on
  the left: psi_{q-1} = F- psi_q with F- = U- diag(1/lambda) U-^+,
  g_L = (D + L F-)^-1, Sigma_L = A_{1,0} g_L A_{0,1}.
When the annulus holds all s modes of a direction, U+ (U-) is square and this
equals the surface Green's function of the decimation exactly; with fewer, the
fast-decaying modes are dropped, as the paper does ("the contribution from fast
decaying modes is negligible").
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import leads


def lead_modes(cell, z):
    """All finite eigenpairs (lambda, u) of (L + lambda D + lambda^2 U) u = 0.

    Companion form on v = [u; lambda u]:  [[0, 1], [-L, -D]] v = lambda [[1, 0], [0, U]] v.
    Returns (lam (2s,), u (s, 2s)) with unit-norm columns u."""
    D, U, L = leads.lead_matrices(cell, z)
    s = D.shape[0]
    I = np.eye(s, dtype=np.complex128)
    Z = np.zeros((s, s), np.complex128)
    A = np.block([[Z, I], [-L, -D]])
    B = np.block([[I, Z], [Z, U]])
    lam, V = sla.eig(A, B)
    ok = np.isfinite(lam)
    lam, V = lam[ok], V[:, ok]
    u = V[:s]
    u = u / np.linalg.norm(u, axis=0)
    return lam, u


def in_annulus(lam, R):
    a = np.abs(lam)
    return (a > 1.0 / R) & (a < R)


def surface_gf(cell, z, side, R=np.inf):
    """Surface Green's function of a lead from its Bloch modes inside the annulus.

    side 'R': bulk to the right (right-going modes, |lambda| < 1);
    side 'L': bulk to the left (left-going modes, |lambda| > 1).
    Returns (g, number of modes used)."""
    D, U, L = leads.lead_matrices(cell, z)
    lam, u = lead_modes(cell, z)
    keep = in_annulus(lam, R)
    if side == "R":
        sel = keep & (np.abs(lam) < 1.0)
        Um, f = u[:, sel], lam[sel]
        F = Um @ np.diag(f) @ np.linalg.pinv(Um)
        g = np.linalg.inv(D + U @ F)
    else:
        sel = keep & (np.abs(lam) > 1.0)
        Um, f = u[:, sel], 1.0 / lam[sel]
        F = Um @ np.diag(f) @ np.linalg.pinv(Um)
        g = np.linalg.inv(D + L @ F)
    return g, int(np.sum(sel))


def self_energies(dev, E, R=np.inf, eta=leads.DEFAULT_ETA):
    """Sigma_L, Sigma_R of a device's leads from their modes (same couplings as
    oracle.leads.self_energies).  Returns (Sigma_L, Sigma_R, info)."""
    left, right = leads.lead_cells(dev)
    z = E + 1j * eta
    gL, mL = surface_gf(left, z, "L", R)
    gR, mR = surface_gf(right, z, "R", R)
    A01 = E * left[3] - left[1]
    AnR = E * right[3] - right[1]
    return A01.conj().T @ gL @ A01, AnR @ gR @ AnR.conj().T, dict(modes_L=mL, modes_R=mR, gL=gL, gR=gR)

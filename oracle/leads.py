"""Lead self-energies by Sancho-Rubio doubling (FP64 oracle, test infrastructure).

The paper names "the standard iterative decimation technique used in NEGF"
for the boundary self-energy (Sec. 3A) without printing its steps; the steps
below are the textbook Sancho / Lopez-Sancho / Rubio doubling written for the
blocks of M = z S - H.

Reading of the paper (it never mentions a broadening):
* ``z = E + i eta`` is used only inside the semi-infinite leads (D, U, L);
  the device and the device-lead couplings are taken at real E, so
  A = E S - H stays Hermitian (Sec. 3B, "complex Hermitian in 1-D and 2-D").
* leads default to periodic copies of the end cells: the left lead repeats
  cell 1 with the cell-1 -> cell-2 coupling, the right lead repeats cell n with
  the cell-(n-1) -> cell-n coupling.
"""
from __future__ import annotations

import numpy as np

DEFAULT_ETA = 1e-10
DEFAULT_TOL = 1e-14
DEFAULT_MAX_ITER = 100


def lead_cells(dev):
    """(H00, H01, S00, S01) of the left and right leads of ``dev``.

    H01 couples lead cell q to q + 1 (left to right) in both leads.
    """
    if dev.lead_L is not None:
        left = tuple(np.asarray(a, np.complex128) for a in dev.lead_L)
    else:
        if dev.n_b < 2:
            raise ValueError("periodic leads need n_b >= 2 (no coupling block to copy)")
        left = (dev.H_diag[0], dev.H_up[0], dev.S_diag[0], dev.S_up[0])
    if dev.lead_R is not None:
        right = tuple(np.asarray(a, np.complex128) for a in dev.lead_R)
    else:
        if dev.n_b < 2:
            raise ValueError("periodic leads need n_b >= 2 (no coupling block to copy)")
        right = (dev.H_diag[-1], dev.H_up[-1], dev.S_diag[-1], dev.S_up[-1])
    return left, right


def lead_matrices(cell, z):
    """Blocks of z S - H for a lead: D (on-site), U (q -> q+1), L (q+1 -> q).

    ``L = z S01^H - H01^H``: with complex z this is *not* U^H.
    """
    H00, H01, S00, S01 = cell
    D = z * S00 - H00
    U = z * S01 - H01
    L = z * S01.conj().T - H01.conj().T
    return D, U, L


def norm1(a):
    """Matrix 1-norm: largest column sum of |a_ij|."""
    return float(np.max(np.sum(np.abs(a), axis=0)))


def sancho_rubio(D, U, L, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER, history=False):
    """Doubling on the semi-infinite chain with blocks (D, U, L).

    One step eliminates every other remaining cell:
      ga = e^-1 a,  gb = e^-1 b
      es_R <- es_R - a gb      (surface cell, bulk to the right)
      es_L <- es_L - b ga      (surface cell, bulk to the left)
      e    <- e - a gb - b ga  (bulk cell)
      a    <- -a ga,  b <- -b gb
    starting from es_R = es_L = e = D, a = U, b = L, until
    max(|a|_1, |b|_1) <= tol |D|_1.  The surface Green's functions are
    g_R = es_R^-1 and g_L = es_L^-1.

    Returns dict(esR, esL, e, iters, converged[, hist]) where ``hist`` lists
    (esR, esL, e) after each step when ``history`` is set.
    """
    e = D.copy()
    esR = D.copy()
    esL = D.copy()
    a = U.copy()
    b = L.copy()
    ref = norm1(D)
    hist = []
    it = 0
    converged = max(norm1(a), norm1(b)) <= tol * ref
    while not converged and it < max_iter:
        ga = np.linalg.solve(e, a)
        gb = np.linalg.solve(e, b)
        agb = a @ gb
        bga = b @ ga
        esR = esR - agb
        esL = esL - bga
        e = e - agb - bga
        a = -(a @ ga)
        b = -(b @ gb)
        it += 1
        if history:
            hist.append((esR.copy(), esL.copy(), e.copy()))
        converged = max(norm1(a), norm1(b)) <= tol * ref
    out = dict(esR=esR, esL=esL, e=e, iters=it, converged=converged)
    if history:
        out["hist"] = hist
    return out


def surface_gf(cell, z, side, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER):
    """Surface Green's function of a semi-infinite lead at complex energy z.

    ``side='R'``: bulk extends to the right of the surface cell;
    ``side='L'``: bulk extends to the left.  Returns (g, iters, converged).
    """
    D, U, L = lead_matrices(cell, z)
    r = sancho_rubio(D, U, L, tol, max_iter)
    es = r["esR"] if side == "R" else r["esL"]
    return np.linalg.inv(es), r["iters"], r["converged"]


def self_energies(dev, E, eta=DEFAULT_ETA, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER):
    """Boundary self-energies of the two leads at real energy E (Eq. negf).

    Sigma_L = A_{1,0} g_L A_{0,1},  Sigma_R = A_{n,n+1} g_R A_{n+1,n},
    with A_{0,1} = E S01 - H01 of the left lead, A_{n,n+1} = E S01 - H01 of the
    right lead (real E) and A_{1,0}, A_{n+1,n} their conjugate transposes.
    Returns (Sigma_L, Sigma_R, info) with the iteration counts in ``info``.
    """
    left, right = lead_cells(dev)
    z = E + 1j * eta
    gL, itL, cL = surface_gf(left, z, "L", tol, max_iter)
    gR, itR, cR = surface_gf(right, z, "R", tol, max_iter)
    A01 = E * left[3] - left[1]
    AnR = E * right[3] - right[1]
    sigma_L = A01.conj().T @ gL @ A01
    sigma_R = AnR @ gR @ AnR.conj().T
    info = dict(iters_L=itL, iters_R=itR, converged=bool(cL and cR), gL=gL, gR=gR)
    return sigma_L, sigma_R, info


def gamma(sigma):
    """Broadening Gamma = i (Sigma - Sigma^H)."""
    return 1j * (sigma - sigma.conj().T)

"""Plain dense definition of the open-boundary solve (FP64 oracle, test infrastructure).

The system is (E S - H - Sigma^RB) c = Inj (Eq. wf) with Sigma^RB non-zero only
in the first and last diagonal blocks, and G^R its inverse (Eq. negf).  The
dense matrix is assembled block by block and solved with LAPACK LU with
partial pivoting; nothing of the block-column recursion is used here, so this
module is the definition the block sweeps must reproduce.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import leads


def assemble_A(dev, E):
    """Dense A = E S - H (N x N) from the device blocks; lower = upper^H."""
    n, s = dev.n_b, dev.s_b
    N = n * s
    A = np.zeros((N, N), np.complex128)
    for i in range(n):
        A[i * s:(i + 1) * s, i * s:(i + 1) * s] = E * dev.S_diag[i] - dev.H_diag[i]
    for i in range(n - 1):
        up = E * dev.S_up[i] - dev.H_up[i]
        A[i * s:(i + 1) * s, (i + 1) * s:(i + 2) * s] = up
        A[(i + 1) * s:(i + 2) * s, i * s:(i + 1) * s] = up.conj().T
    return A


def system_matrix(dev, E, sigma_L, sigma_R):
    """M = A - Sigma_L (+) 0 (+) ... (+) Sigma_R."""
    s = dev.s_b
    M = assemble_A(dev, E)
    M[:s, :s] -= sigma_L
    M[-s:, -s:] -= sigma_R
    return M


def full_injection(inj_rows, n, s):
    """Inj (N x n_inj) from its non-zero rows b' (2s x n_inj): block 1 then block n."""
    inj_rows = np.asarray(inj_rows)
    N = n * s
    b = np.zeros((N, inj_rows.shape[1]), np.complex128)
    b[:s] += inj_rows[:s]
    b[-s:] += inj_rows[s:]
    return b


def corners(lu, n, s):
    """G_11, G_1n, G_n1, G_nn of M^-1 from an LU factorisation of M."""
    N = n * s
    E1 = np.zeros((N, s), np.complex128)
    E1[:s] = np.eye(s)
    En = np.zeros((N, s), np.complex128)
    En[-s:] = np.eye(s)
    c1 = sla.lu_solve(lu, E1)
    cn = sla.lu_solve(lu, En)
    return dict(G11=c1[:s], Gn1=c1[-s:], G1n=cn[:s], Gnn=cn[-s:], col1=c1, coln=cn)


def caroli(sigma_L, sigma_R, G1n):
    """Tr[Gamma_L G_1n Gamma_R G_1n^H] (complex; its real part is T)."""
    gl = leads.gamma(sigma_L)
    gr = leads.gamma(sigma_R)
    return complex(np.trace(gl @ G1n @ gr @ G1n.conj().T))


def solve_point(dev, E, inj_rows=None, eta=leads.DEFAULT_ETA, tol=leads.DEFAULT_TOL,
                max_iter=leads.DEFAULT_MAX_ITER, sigmas=None):
    """Everything the hot path produces for one (E, k) point, by definition.

    Returns dict with Sigma_L, Sigma_R, the four corners of G = M^-1, the
    transmission T (real part of the Caroli trace) and its imaginary part,
    T_RL (the reverse trace with G_n1), and ``x = M^-1 Inj`` when
    ``inj_rows`` (2s x n_inj) is given.
    """
    n, s = dev.n_b, dev.s_b
    if sigmas is None:
        sL, sR, info = leads.self_energies(dev, E, eta, tol, max_iter)
    else:
        sL, sR = sigmas
        info = {}
    M = system_matrix(dev, E, sL, sR)
    lu = sla.lu_factor(M)
    c = corners(lu, n, s)
    tr = caroli(sL, sR, c["G1n"])
    tr_rl = caroli(sR, sL, c["Gn1"])
    out = dict(sigma_L=sL, sigma_R=sR, T=tr.real, T_imag=tr.imag, T_RL=tr_rl.real,
               M=M, info=info, **c)
    if inj_rows is not None:
        b = full_injection(inj_rows, n, s)
        out["x"] = sla.lu_solve(lu, b)
        out["inj_full"] = b
    return out


def bond_currents(dev, E, x):
    """J_i = 2 Im Tr[x_i^H (H_{i,i+1} - E S_{i,i+1}) x_{i+1}], i = 1..n-1.

    For a solution of the open system with injection from one lead, the
    current carried between neighbouring cells is the same for every i.
    """
    n, s = dev.n_b, dev.s_b
    J = []
    for i in range(n - 1):
        xi = x[i * s:(i + 1) * s]
        xj = x[(i + 1) * s:(i + 2) * s]
        hop = dev.H_up[i] - E * dev.S_up[i]
        J.append(2.0 * np.imag(np.trace(xi.conj().T @ hop @ xj)))
    return np.asarray(J)


def residual(M, x, b):
    """||M x - b||_F / ||b||_F."""
    return float(np.linalg.norm(M @ x - b) / np.linalg.norm(b))


def backward_error(M, x, b):
    """Normwise backward error in Frobenius norms (Rigal and Gaches):
    ||M x - b|| / (||M|| ||x|| + ||b||), the smallest eps for which
    (M + dM) x = b + db with ||dM|| <= eps ||M|| and ||db|| <= eps ||b||."""
    r = M @ x - b
    return float(np.linalg.norm(r) / (np.linalg.norm(M) * np.linalg.norm(x) + np.linalg.norm(b)))


def rel_T_err(T, T_ref):
    """|T - T_ref| / max(1, |T_ref|): a relative error that stays defined in gaps."""
    return abs(T - T_ref) / max(1.0, abs(T_ref))


def ldos(dev, E, eta=leads.DEFAULT_ETA, tol=leads.DEFAULT_TOL, max_iter=leads.DEFAULT_MAX_ITER, sigmas=None):
    """Local density of states per block, rho_i = -Im Tr[G_ii] / pi, from the
    dense inverse G = (E S - H - Sigma)^-1 of the open system (Eq. negf: G^R is
    the inverse of the boundary-corrected matrix of Eq. wf).  The blocks' traces
    are the spectral weight the paper's observables (charge and current
    densities, Sec. 2B) are integrated from.  Returns an array of n_b values."""
    n, s = dev.n_b, dev.s_b
    if sigmas is None:
        sL, sR, _ = leads.self_energies(dev, E, eta, tol, max_iter)
    else:
        sL, sR = sigmas
    G = np.linalg.inv(system_matrix(dev, E, sL, sR))
    return np.array([-np.trace(G[i * s:(i + 1) * s, i * s:(i + 1) * s]).imag / np.pi for i in range(n)])

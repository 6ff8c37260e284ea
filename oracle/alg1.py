"""Algorithm 1 and the SMW steps written in the paper's order (oracle, test infrastructure).

Used by the pins that check the readings the block sweeps rely on:

* Algorithm 1 solves (A_ii - A_{i,i+1} X_{i+1}) X_i = A_{i,i-1} for i = n_B..1
  with X_{n_B+1} = 0, then Q_i = -X_i Q_{i-1} with Q_0 = -1.  The paper leaves
  A_{1,0} undefined; the reading is A_{1,0} := 1, which makes Q_1 = X_1 the
  (1,1) block of A^-1 and Q_i = [A^-1]_{i,1}.
* The last block column follows "similarly" (Sec. 3B): the same recursion on
  the block-reversed matrix, i.e. a forward elimination with A_{n,n+1} := 1.
* Steps 1-4 of Eq. x with Sigma^RB = B C and T = A - B C:
  Q = A^-1 B, y = A^-1 b, (1 - C Q) z = C y, x = y + Q z; equivalently
  x = Q (b' + z) with y = Q b'.
"""
from __future__ import annotations

import numpy as np


def _blk(dev, E):
    n = dev.n_b
    Ad = [E * dev.S_diag[i] - dev.H_diag[i] for i in range(n)]
    Au = [E * dev.S_up[i] - dev.H_up[i] for i in range(n - 1)]
    return Ad, Au


def first_block_column(dev, E):
    """[A^-1]_{i,1}, i = 1..n, by Algorithm 1 (list of s x s blocks)."""
    n, s = dev.n_b, dev.s_b
    Ad, Au = _blk(dev, E)
    I = np.eye(s, dtype=np.complex128)
    X = [None] * (n + 2)
    X[n + 1] = np.zeros((s, s), np.complex128)
    for i in range(n, 0, -1):
        Aii = Ad[i - 1]
        Aup = Au[i - 1] if i < n else np.zeros((s, s), np.complex128)
        Alo = Au[i - 2].conj().T if i > 1 else I          # A_{1,0} := 1
        X[i] = np.linalg.solve(Aii - Aup @ X[i + 1], Alo)
    Q = [-I]
    for i in range(1, n + 1):
        Q.append(-X[i] @ Q[i - 1])
    return Q[1:]


def last_block_column(dev, E):
    """[A^-1]_{i,n}, i = 1..n: Algorithm 1 mirrored (A_{n,n+1} := 1)."""
    n, s = dev.n_b, dev.s_b
    Ad, Au = _blk(dev, E)
    I = np.eye(s, dtype=np.complex128)
    Y = [None] * (n + 2)
    Y[0] = np.zeros((s, s), np.complex128)
    for i in range(1, n + 1):
        Aii = Ad[i - 1]
        Alo = Au[i - 2].conj().T if i > 1 else np.zeros((s, s), np.complex128)
        Aup = Au[i - 1] if i < n else I                    # A_{n,n+1} := 1
        Y[i] = np.linalg.solve(Aii - Alo @ Y[i - 1], Aup)
    P = [None] * (n + 2)
    P[n + 1] = -I
    for i in range(n, 0, -1):
        P[i] = -Y[i] @ P[i + 1]
    return P[1:n + 1]


def smw_solve(dev, E, sigma_L, sigma_R, inj_rows):
    """Steps 1-4 of Eq. x: returns (x, R, g, G_b) for T = A - B C.

    ``g`` is the 2s x 2s corner matrix B^T A^-1 B and ``G_b = g R^-1`` the
    corners of (A - BC)^-1.
    """
    n, s = dev.n_b, dev.s_b
    Qf = first_block_column(dev, E)
    Ql = last_block_column(dev, E)
    Q = np.zeros((n * s, 2 * s), np.complex128)
    for i in range(n):
        Q[i * s:(i + 1) * s, :s] = Qf[i]
        Q[i * s:(i + 1) * s, s:] = Ql[i]
    g = np.vstack([Q[:s], Q[-s:]])                          # B^T Q
    Sb = np.zeros((2 * s, 2 * s), np.complex128)
    Sb[:s, :s] = sigma_L
    Sb[s:, s:] = sigma_R
    R = np.eye(2 * s) - Sb @ g                              # 1 - C Q, C = Sb B^T
    y = Q @ inj_rows                                        # y = A^-1 b = Q b'
    Cy = Sb @ np.vstack([y[:s], y[-s:]])
    z = np.linalg.solve(R, Cy)
    x = Q @ (inj_rows + z)                                  # x = y + Q z
    Gb = g @ np.linalg.inv(R)
    return x, R, g, Gb

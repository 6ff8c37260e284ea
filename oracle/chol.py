"""Rank-revealing pivoted Cholesky of a Hermitian PSD matrix (oracle, test infrastructure).

Gamma_R = V V^H gives the injection Inj = [0; V] whose first block of the
solution x_1 = G_1n V carries the transmission T = Tr[x_1^H Gamma_L x_1]
(the same quantity as the Caroli trace, with one column per open channel).

Pivot: the largest remaining diagonal entry, lowest index on ties; stop when
it falls to ``rtol`` times the largest initial diagonal entry.
"""
from __future__ import annotations

import numpy as np


def pivoted_cholesky(G, rtol=1e-10):
    """Return V (s x r) with G ~= V V^H and the pivot order."""
    G = np.asarray(G, np.complex128)
    s = G.shape[0]
    d = np.real(np.diag(G)).copy()
    dmax0 = float(np.max(d)) if s else 0.0
    V = np.zeros((s, s), np.complex128)
    piv = []
    r = 0
    if dmax0 <= 0.0:
        return V[:, :0], piv
    while r < s:
        p = int(np.argmax(d))
        if d[p] <= rtol * dmax0:
            break
        col = G[:, p] - V[:, :r] @ V[p, :r].conj()
        col = col / np.sqrt(d[p])
        V[:, r] = col
        d = d - np.abs(col) ** 2
        d[p] = 0.0
        piv.append(p)
        r += 1
    return V[:, :r], piv

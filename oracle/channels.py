"""Open-channel count of a lead (FP64 oracle, test infrastructure).

The lead's Bloch modes psi_q = lambda^q u solve the one-neighbour case of
Eq. bound:  (H10 - E S10) + (H00 - E S00) lambda + (H01 - E S01) lambda^2 = 0,
with H10 = H01^H, S10 = S01^H.  Propagating modes have |lambda| = 1; half of
them move to the right.  A perfect periodic wire therefore transmits exactly
(number of unimodular lambda) / 2 at a real energy away from band edges.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def bloch_factors(cell, E):
    """All finite eigenvalues lambda of the quadratic pencil (companion form)."""
    H00, H01, S00, S01 = cell
    s = H00.shape[0]
    C2 = H01 - E * S01
    C1 = H00 - E * S00
    C0 = H01.conj().T - E * S01.conj().T
    I = np.eye(s)
    Z = np.zeros((s, s))
    A = np.block([[Z, I], [-C0, -C1]])
    B = np.block([[I, Z], [Z, C2]])
    lam = sla.eig(A, B, right=False)
    return lam[np.isfinite(lam)]


def open_channels(cell, E, tol=1e-8):
    """Number of right-moving propagating modes: #{|lambda| = 1} / 2."""
    lam = bloch_factors(cell, E)
    n_unit = int(np.sum(np.abs(np.abs(lam) - 1.0) < tol))
    return n_unit // 2, n_unit

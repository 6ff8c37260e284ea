"""Seeded synthetic inputs for the open-boundary block-tridiagonal problem.

This module only builds random matrices and grids.  It holds no step of the
solver's arithmetic (no self-energy, no factorisation, no transmission), so
that both the FP64 CPU oracle and the CUDA library can be fed from it without
sharing any of the method.

Shapes follow the workloads of the paper's transport runs (Sec. 2, Eq. wf;
Sec. 3B): a device of ``n_b`` diagonal blocks of size ``s_b`` with Hermitian
diagonal blocks, nearest-block couplings and a positive-definite overlap.
Every array is complex128 and C-contiguous, blocks row-major.

Recipe (each choice stated once, used everywhere):

* ``G`` = N(0,1) + i N(0,1), iid per entry.
* ``H_ii = (G + G^H) / 2``; couplings ``H_{i,i+1} = coupling * G'``
  (a general complex block).
* ``S_ii = I + s_pert * (G'' + G''^H) / 2 / (4 sqrt(s))`` and
  ``S_{i,i+1} = s_pert * G''' / (4 sqrt(s))``: the ``4 sqrt(s)`` divisor keeps
  the periodic overlap S(k) above 0.5 for s_pert <= 0.1.
* optional band mask ``|a - b| <= band`` on every block (the "sparse-banded"
  nanowire-like inputs keep about 10 % of each block at s = 512, band = 25).
* optional transverse momentum: ``H(k) = H0 + W e^{ik} + W^H e^{-ik}`` per
  block, with ``W`` a seeded complex block scaled by ``w_scale`` times the
  block's own scale (same construction for S with the S scale).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Device",
    "make_device",
    "make_injection",
    "energy_grid",
    "K_POINTS_4",
    "decoupled_wire",
    "periodic_wire",
    "uneven_points",
]

K_POINTS_4 = (0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4)


def _cgauss(rng: np.random.Generator, shape) -> np.ndarray:
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _band(s: int, band: int | None) -> np.ndarray | None:
    if band is None or band >= s:
        return None
    idx = np.arange(s)
    return (np.abs(idx[:, None] - idx[None, :]) <= band).astype(np.float64)


@dataclass
class Device:
    """Blocks of one device Hamiltonian at one transverse momentum.

    ``H_diag``/``S_diag``: (n_b, s, s); ``H_up``/``S_up``: (n_b - 1, s, s) with
    ``H_up[i]`` the block coupling cell i to cell i + 1 (0-based).  The lower
    blocks are the conjugate transposes.  ``lead_L``/``lead_R`` are ``None``
    (leads are periodic copies of the end cells) or a tuple
    ``(H00, H01, S00, S01)`` of s x s blocks, H01 coupling lead cell q to q + 1.
    """

    H_diag: np.ndarray
    H_up: np.ndarray
    S_diag: np.ndarray
    S_up: np.ndarray
    lead_L: tuple | None = None
    lead_R: tuple | None = None
    k: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_b(self) -> int:
        return self.H_diag.shape[0]

    @property
    def s_b(self) -> int:
        return self.H_diag.shape[1]


def make_device(
    n_b: int,
    s_b: int,
    seed: int,
    *,
    s_pert: float = 0.05,
    coupling: float = 0.5,
    band: int | None = None,
    k_points=(0.0,),
    w_scale: float = 0.0,
) -> list[Device]:
    """Seeded device blocks, one :class:`Device` per entry of ``k_points``.

    ``w_scale = 0`` gives k-independent blocks (the single-point workloads).
    """
    if n_b < 1 or s_b < 1:
        raise ValueError("n_b and s_b must be positive")
    rng = np.random.default_rng(seed)
    s = s_b
    mask = _band(s, band)
    snorm = s_pert / (4.0 * math.sqrt(s))

    def masked(a):
        return a if mask is None else a * mask

    H0d = np.empty((n_b, s, s), np.complex128)
    S0d = np.empty((n_b, s, s), np.complex128)
    for i in range(n_b):
        g = _cgauss(rng, (s, s))
        H0d[i] = masked((g + g.conj().T) / 2)
        g = _cgauss(rng, (s, s))
        S0d[i] = np.eye(s) + masked(snorm * (g + g.conj().T) / 2)
    H0u = np.empty((max(n_b - 1, 0), s, s), np.complex128)
    S0u = np.empty_like(H0u)
    for i in range(n_b - 1):
        H0u[i] = masked(coupling * _cgauss(rng, (s, s)))
        S0u[i] = masked(snorm * _cgauss(rng, (s, s)))

    out = []
    if w_scale == 0.0:
        for k in k_points:
            out.append(Device(H0d.copy(), H0u.copy(), S0d.copy(), S0u.copy(), k=float(k),
                              meta=dict(seed=seed, band=band, s_pert=s_pert)))
        return out

    # transverse-momentum terms, drawn after the k-independent part
    Wd = np.stack([masked(w_scale * 0.5 * _cgauss(rng, (s, s))) for _ in range(n_b)])
    Wu1 = np.stack([masked(w_scale * coupling * 0.5 * _cgauss(rng, (s, s))) for _ in range(n_b - 1)]) \
        if n_b > 1 else np.zeros((0, s, s), np.complex128)
    Wu2 = np.stack([masked(w_scale * coupling * 0.5 * _cgauss(rng, (s, s))) for _ in range(n_b - 1)]) \
        if n_b > 1 else np.zeros((0, s, s), np.complex128)
    Vd = np.stack([masked(w_scale * snorm * 0.5 * _cgauss(rng, (s, s))) for _ in range(n_b)])
    Vu1 = np.stack([masked(w_scale * snorm * 0.5 * _cgauss(rng, (s, s))) for _ in range(n_b - 1)]) \
        if n_b > 1 else np.zeros((0, s, s), np.complex128)
    Vu2 = np.stack([masked(w_scale * snorm * 0.5 * _cgauss(rng, (s, s))) for _ in range(n_b - 1)]) \
        if n_b > 1 else np.zeros((0, s, s), np.complex128)
    for k in k_points:
        ep, em = np.exp(1j * k), np.exp(-1j * k)
        Hd = H0d + Wd * ep + np.conj(np.swapaxes(Wd, 1, 2)) * em
        Sd = S0d + Vd * ep + np.conj(np.swapaxes(Vd, 1, 2)) * em
        Hu = H0u + Wu1 * ep + Wu2 * em
        Su = S0u + Vu1 * ep + Vu2 * em
        out.append(Device(Hd, Hu, Sd, Su, k=float(k),
                          meta=dict(seed=seed, band=band, s_pert=s_pert, w_scale=w_scale)))
    return out


def make_injection(s_b: int, n_inj: int, seed: int, n_pts: int = 1) -> np.ndarray:
    """Seeded injection rows ``b'``: (n_pts, 2 s_b, n_inj) complex128.

    Rows 0..s-1 act on the first block row, rows s..2s-1 on the last one
    (the only non-zero rows of Inj, Sec. 3B).
    """
    rng = np.random.default_rng(seed)
    return _cgauss(rng, (n_pts, 2 * s_b, n_inj)) / math.sqrt(2.0)


def energy_grid(n_e: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform grid including both ends: lo + (hi - lo) j / (n_e - 1)."""
    if n_e == 1:
        return np.array([0.5 * (lo + hi)])
    return lo + (hi - lo) * np.arange(n_e) / (n_e - 1)


def decoupled_wire(s_b: int, n_b: int, t: float, seed: int):
    """A wire of ``s_b`` independent 1-D chains in a rotated basis.

    ``H00 = V diag(eps) V^H``, ``H01 = t I``, ``S = I``; returns the
    :class:`Device` (device cells equal to lead cells) and ``eps``.
    """
    rng = np.random.default_rng(seed)
    eps = rng.uniform(-1.5, 1.5, s_b)
    q, _ = np.linalg.qr(_cgauss(rng, (s_b, s_b)))
    H00 = (q * eps) @ q.conj().T
    H00 = (H00 + H00.conj().T) / 2
    H01 = t * np.eye(s_b, dtype=np.complex128)
    I = np.eye(s_b, dtype=np.complex128)
    dev = Device(
        np.stack([H00] * n_b), np.stack([H01] * (n_b - 1)),
        np.stack([I] * n_b), np.stack([np.zeros_like(I)] * (n_b - 1)),
    )
    return dev, eps


def periodic_wire(s_b: int, n_b: int, seed: int, coupling: float = 0.5, s_pert: float = 0.05):
    """A perfect periodic wire with general (H00, H01, S00, S01) cells."""
    cell = make_device(2, s_b, seed, coupling=coupling, s_pert=s_pert)[0]
    H00, H01, S00, S01 = cell.H_diag[0], cell.H_up[0], cell.S_diag[0], cell.S_up[0]
    dev = Device(
        np.stack([H00] * n_b), np.stack([H01] * (n_b - 1)),
        np.stack([S00] * n_b), np.stack([S01] * (n_b - 1)),
    )
    return dev, (H00, H01, S00, S01)


def uneven_points(n_pts: int, seed: int, s_choices=(256, 384, 512), n_choices=(32, 64, 128),
                  k_points=K_POINTS_4):
    """(s_b, n_b, E, k) tuples drawn uniformly for the uneven-batch workload."""
    rng = np.random.default_rng(seed)
    s = rng.choice(np.asarray(s_choices), n_pts)
    n = rng.choice(np.asarray(n_choices), n_pts)
    E = rng.uniform(-1.0, 1.0, n_pts)
    k = rng.choice(np.asarray(k_points), n_pts)
    return [(int(s[i]), int(n[i]), float(E[i]), float(k[i])) for i in range(n_pts)]

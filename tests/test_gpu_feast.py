"""Contour-integral (FEAST) open boundary conditions (Sec. 3A, Eq. bound,
Eq. feast) on the GPU against the oracle's mode-based self-energies.

The oracle takes the lead's Bloch modes from a dense generalized eigensolver
(the plain definition of what the contour integral and Rayleigh-Ritz step
compute); with an annulus holding all modes the result also equals the
decimation's, by an independent route.  Bars: Sigma within 1e-9 (relative
Frobenius; the modes' eigenvector matrix enters through its condition
number), and T and x of the whole solve at the usual parity bar when every
mode is captured."""
import math

import numpy as np
import pytest

import synth
from oracle import dense, feast, leads

from test_gpu_parity import check_point, rel, run_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def feast_sigmas(ss, devs, Es, **cfg):
    h = ss.Handle(n_b_max=max(d.n_b for d in devs), s_b_max=max(d.s_b for d in devs), max_points=len(Es), max_inj=1,
                  obc=ss.SS_OBC_FEAST, **cfg)
    try:
        for k, d in enumerate(devs):
            h.set_device(k, d)
        sL, sR, it, st, rc = h.self_energy(Es, list(range(len(devs))))
    finally:
        h.close()
    return sL, sR, np.asarray(st)


@pytest.mark.parametrize("s", [6, 12, 24])
def test_feast_sigma_equals_oracle_modes_and_decimation(ss, s):
    dev = synth.make_device(3, s, seed=200 + s)[0]
    Es = [-0.4, 0.7, 2.5]
    sL, sR, st = feast_sigmas(ss, [dev] * 3, Es, feast_radius=1e3, feast_points=24)
    assert np.all(st == 0)
    for p, E in enumerate(Es):
        fL, fR, info = feast.self_energies(dev, E, R=1e3)
        dL, dR, _ = leads.self_energies(dev, E)
        assert info["modes_L"] == s and info["modes_R"] == s
        assert rel(sL[p], fL) < 1e-9 and rel(sR[p], fR) < 1e-9, (rel(sL[p], fL), rel(sR[p], fR))
        assert rel(sL[p], dL) < 1e-9 and rel(sR[p], dR) < 1e-9


def test_feast_reduced_annulus_matches_oracle(ss):
    """A smaller annulus drops the fast-decaying modes; the GPU drops the same
    ones as the oracle (same R), so their self-energies agree."""
    s = 12
    dev = synth.make_device(3, s, seed=212)[0]
    E = 0.3
    # the radius: the widest gap in log |lambda| above the unit circle, so both
    # circles (R and 1/R) pass between eigenvalues and a few modes fall outside
    mods = []
    for side in (0, 1):
        lam, _ = feast.lead_modes(leads.lead_cells(dev)[side], E + 1j * leads.DEFAULT_ETA)
        mods.append(np.abs(lam))
    a = np.sort(np.concatenate([np.concatenate(mods), 1.0 / np.concatenate(mods)]))
    la = np.log(a[a > 1.2])
    gaps = np.diff(la)
    i = int(np.argmax(gaps[:-1]))       # not beyond the largest modulus
    R = float(np.exp(0.5 * (la[i] + la[i + 1])))
    assert np.min(np.abs(np.log(a) - np.log(R))) > 0.1
    sL, sR, st = feast_sigmas(ss, [dev], [E], feast_radius=R, feast_points=32)
    fL, fR, info = feast.self_energies(dev, E, R=R)
    assert info["modes_L"] + info["modes_R"] < 2 * s  # modes were dropped
    assert rel(sR[0], fR) < 1e-8 and rel(sL[0], fL) < 1e-8


def test_feast_chain_closed_form(ss):
    eps0, t = 0.2, -0.7
    chain = synth.Device(np.full((4, 1, 1), eps0, np.complex128), np.full((3, 1, 1), t, np.complex128),
                         np.ones((4, 1, 1), np.complex128), np.zeros((3, 1, 1), np.complex128))
    ks = [0.4, 1.3, 2.2]
    Es = [eps0 + 2 * t * math.cos(k) for k in ks]
    sL, sR, st = feast_sigmas(ss, [chain] * 3, Es, feast_radius=10.0)
    for p, k in enumerate(ks):
        assert abs(complex(sR[p][0, 0]) - t * np.exp(1j * k)) < 1e-7
        assert abs(complex(sL[p][0, 0]) - t * np.exp(1j * k)) < 1e-7


@pytest.mark.parametrize("prec", [0, 3])
def test_feast_pipeline_transmission_and_wave_functions(ss, prec):
    """The whole solve with the contour-integral self-energies: x and T at the
    parity bar of the decimation path (all modes inside the annulus)."""
    dev = synth.make_device(5, 16, seed=230)[0]
    Es = [0.15, -0.55]
    inj = [synth.make_injection(16, 3, seed=231 + i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj, precision=prec, obc=ss.SS_OBC_FEAST, feast_radius=1e3, feast_points=24)
    assert np.all(np.asarray(r["st_T"]) == 0)
    for p in range(2):
        check_point(r, p, dev, Es[p], inj[p])

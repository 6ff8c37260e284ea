"""The next rows of the scope: transmission-only (memory-lean) solves,
partitioned sweeps merged by one boundary system, and the density of states.

* Transmission-only mode keeps the corner blocks of the inverse as running
  products instead of both block columns; its T must meet the parity bar of
  the full solve (1e-10, or 20 x the oracle's one-ulp sensitivity), and a
  memory-lean handle must fit more points in less memory.
* Partitioned sweeps (Sec. 3B, Fig. pp): each partition's first and last
  block columns, merged with the leads in one Sherman-Morrison-Woodbury system;
  T, Sigma and x against the oracle for 2..4 partitions, ragged partitions and
  partitions of a single block, FP64 and mixed paths.
* Density of states rho_i = -Im Tr[G_ii] / pi of the open system: against the
  dense oracle's diagonal blocks, and against closed forms (perfect chain,
  decoupled wire).
"""
import math

import numpy as np
import pytest

import synth
from oracle import dense

from test_gpu_parity import TOL, check_point, noise_floor, rel, run_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def transmission_only(ss, devs, Es, **cfg):
    n_max = max(d.n_b for d in devs)
    s_max = max(d.s_b for d in devs)
    h = ss.Handle(n_b_max=n_max, s_b_max=s_max, max_points=cfg.pop("max_points", len(Es)), max_inj=1, **cfg)
    try:
        for k, d in enumerate(devs):
            h.set_device(k, d)
        T, err, st, rc = h.transmission(Es, list(range(len(devs))))
    finally:
        h.close()
    return np.asarray(T), np.asarray(st)


# --------------------------------------------------- transmission-only mode
@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("n_b,s_b", [(16, 32), (5, 70), (1, 12), (2, 33)])
def test_transmission_only_matches_oracle(ss, prec, n_b, s_b):
    if n_b == 1:
        cell = synth.make_device(2, s_b, seed=8)[0]
        lead = (cell.H_diag[0], cell.H_up[0], cell.S_diag[0], cell.S_up[0])
        dev = synth.Device(cell.H_diag[:1].copy(), np.zeros((0, s_b, s_b), np.complex128), cell.S_diag[:1].copy(),
                           np.zeros((0, s_b, s_b), np.complex128), lead_L=lead, lead_R=lead)
    else:
        dev = synth.make_device(n_b, s_b, seed=50 + s_b)[0]
    Es = [0.3, -0.45]
    T, st = transmission_only(ss, [dev, dev], Es, precision=prec)
    assert np.all(st == 0)
    for p, E in enumerate(Es):
        ref = dense.solve_point(dev, E)
        bar = max(TOL, 20.0 * noise_floor(dev, E, None, ref)["T"])
        assert dense.rel_T_err(float(T[p]), ref["T"]) < bar


def test_memory_lean_handle_is_smaller_and_agrees(ss):
    """A memory-lean handle fits the same transmissions in a fraction of the
    device memory of a full one (no block columns are stored)."""
    import torch
    dev = synth.make_device(48, 64, seed=61)[0]
    Es = [0.2, -0.3, 0.6, -0.8]
    used = {}
    T = {}
    for lean in (0, 1):
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        h = ss.Handle(n_b_max=48, s_b_max=64, max_points=4, max_inj=1, memory_lean=lean)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        try:
            h.set_device(0, dev)
            Tv, _, st, _ = h.transmission(Es, [0] * 4)
        finally:
            h.close()
        assert np.all(np.asarray(st) == 0)
        used[lean] = free0 - free1
        T[lean] = np.asarray(Tv)
    assert used[1] < 0.5 * used[0], used  # 51 s^2 against (2 n_b + 45) s^2 per point
    for p, E in enumerate(Es):
        ref = dense.solve_point(dev, E)
        assert dense.rel_T_err(float(T[1][p]), ref["T"]) < max(TOL, 20.0 * noise_floor(dev, E, None, ref)["T"])
    # wave functions on a lean handle: refused for lack of room, not silently wrong
    h = ss.Handle(n_b_max=48, s_b_max=64, max_points=1, max_inj=2, memory_lean=1)
    try:
        h.set_device(0, dev)
        with pytest.raises(ss.SSError) as e:
            h.solve([0.2], [0], [synth.make_injection(64, 2, seed=1)[0]])
        assert e.value.code == ss.SS_ERR_OOM
    finally:
        h.close()


# -------------------------------------------------------- partitioned sweeps
@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("n_b,s_b,parts", [(8, 40, 2), (7, 33, 3), (3, 24, 3), (9, 17, 4), (16, 32, 2)])
def test_partitioned_sweeps_match_oracle(ss, prec, n_b, s_b, parts):
    dev = synth.make_device(n_b, s_b, seed=70 + n_b + s_b)[0]
    Es = [0.15, -0.6]
    inj = [synth.make_injection(s_b, 3, seed=80 + i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj, precision=prec, partitions=parts)
    assert np.all(np.asarray(r["st_T"]) == 0)
    for p in range(2):
        check_point(r, p, dev, Es[p], inj[p])
    T, st = transmission_only(ss, [dev, dev], Es, precision=prec, partitions=parts)
    assert np.all(st == 0)
    for p in range(2):
        assert dense.rel_T_err(float(T[p]), float(r["T"][p])) < 1e-10


def test_partitioned_uneven_batch(ss):
    """Points of different (n_b, s_b) split into partitions of different lengths in the same launches."""
    devs = [synth.make_device(6, 40, seed=91)[0], synth.make_device(11, 24, seed=92)[0],
            synth.make_device(2, 50, seed=93)[0]]
    Es = [0.2, -0.7, 0.55]
    inj = [synth.make_injection(d.s_b, 2, seed=95 + i)[0] for i, d in enumerate(devs)]
    r = run_points(ss, devs, Es, inj, partitions=3)
    for p, d in enumerate(devs):
        check_point(r, p, d, Es[p], inj[p])


def test_partitions_shorten_the_sweep(ss):
    """Two partitions halve the sequential sweep steps of a long device: fewer
    launches per solve for the same result."""
    dev = synth.make_device(32, 16, seed=97)[0]
    a = run_points(ss, [dev], [0.3], partitions=1)
    b = run_points(ss, [dev], [0.3], partitions=2)
    assert dense.rel_T_err(float(b["T"][0]), float(a["T"][0])) < 1e-10
    assert b["launches"] < a["launches"], (a["launches"], b["launches"])


# --------------------------------------------------------- density of states
def dos_of(ss, devs, Es, **cfg):
    n_max = max(d.n_b for d in devs)
    s_max = max(d.s_b for d in devs)
    h = ss.Handle(n_b_max=n_max, s_b_max=s_max, max_points=cfg.pop("max_points", len(Es)), max_inj=1, **cfg)
    try:
        for k, d in enumerate(devs):
            h.set_device(k, d)
        rho, st, rc = h.dos(Es, list(range(len(devs))))
    finally:
        h.close()
    return [np.asarray(x) for x in rho], np.asarray(st)


def ldos_sensitivity(dev, E, ref):
    rng = np.random.default_rng(1234)
    out = 0.0
    for _ in range(2):
        d2 = synth.Device(dev.H_diag * (1 + 2.0 ** -52 * rng.standard_normal(dev.H_diag.shape)),
                          dev.H_up * (1 + 2.0 ** -52 * rng.standard_normal(dev.H_up.shape)),
                          dev.S_diag, dev.S_up, lead_L=dev.lead_L, lead_R=dev.lead_R)
        out = max(out, rel(dense.ldos(d2, E), ref))
    return out


@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("n_b,s_b", [(16, 32), (5, 70), (2, 33), (9, 17)])
def test_dos_matches_dense_oracle(ss, prec, n_b, s_b):
    dev = synth.make_device(n_b, s_b, seed=100 + s_b)[0]
    Es = [0.3, -0.45]
    rho, st = dos_of(ss, [dev, dev], Es, precision=prec)
    assert np.all(st == 0)
    for p, E in enumerate(Es):
        ref = dense.ldos(dev, E)
        bar = max(TOL, 20.0 * ldos_sensitivity(dev, E, ref))
        assert rho[p].shape == (n_b,)
        assert rel(rho[p], ref) < bar, (rel(rho[p], ref), bar)


def test_dos_single_block_and_uneven_batch(ss):
    cell = synth.make_device(2, 12, seed=8)[0]
    lead = (cell.H_diag[0], cell.H_up[0], cell.S_diag[0], cell.S_up[0])
    d1 = synth.Device(cell.H_diag[:1].copy(), np.zeros((0, 12, 12), np.complex128), cell.S_diag[:1].copy(),
                      np.zeros((0, 12, 12), np.complex128), lead_L=lead, lead_R=lead)
    devs = [d1, synth.make_device(11, 20, seed=111)[0], synth.make_device(4, 48, seed=112)[0]]
    Es = [0.05, 0.4, -0.2]
    rho, st = dos_of(ss, devs, Es)
    assert np.all(st == 0)
    for p, d in enumerate(devs):
        ref = dense.ldos(d, Es[p])
        assert rel(rho[p], ref) < max(TOL, 20.0 * ldos_sensitivity(d, Es[p], ref))


def test_dos_closed_forms_on_gpu(ss):
    """Perfect chain: 1 / (pi sqrt(4t^2 - (E-eps0)^2)) on every site; decoupled
    wire: the sum of the in-band chains' densities in every cell."""
    eps0, t = 0.2, -0.7
    chain = synth.Device(np.full((5, 1, 1), eps0, np.complex128), np.full((4, 1, 1), t, np.complex128),
                         np.ones((5, 1, 1), np.complex128), np.zeros((4, 1, 1), np.complex128))
    ks = [0.5, 1.4, 2.6]
    Es = [eps0 + 2 * t * math.cos(k) for k in ks]
    rho, st = dos_of(ss, [chain] * 3, Es)
    for p, E in enumerate(Es):
        expect = 1.0 / (math.pi * math.sqrt(4 * t * t - (E - eps0) ** 2))
        assert np.allclose(rho[p], expect, rtol=1e-8, atol=0)
    s, tw = 16, -0.8
    wire, eps = synth.decoupled_wire(s, 6, tw, seed=5)
    Ew = []
    for E in np.linspace(-2.0, 2.0, 7):
        edges = np.concatenate([eps - 2 * abs(tw), eps + 2 * abs(tw)])
        if np.min(np.abs(E - edges)) > 0.05:
            Ew.append(float(E))
    rho, st = dos_of(ss, [wire] * len(Ew), Ew)
    for p, E in enumerate(Ew):
        inb = np.abs(E - eps) < 2 * abs(tw)
        expect = float(np.sum(1.0 / (np.pi * np.sqrt(4 * tw * tw - (E - eps[inb]) ** 2))))
        assert np.allclose(rho[p], expect, rtol=1e-7, atol=1e-9)


# ------------------------------------------- Hermitian LDL^H of the sweep blocks
def below_spectrum(dev, margins):
    """Energies below the lowest eigenvalue of the closed device (H, S): there
    A = E S - H is negative definite, and so is every Schur complement D_i."""
    import scipy.linalg as sla
    A0 = dense.assemble_A(dev, 0.0)          # -H
    A1 = dense.assemble_A(dev, 1.0) - A0     # S
    lo = sla.eigh(-A0, A1, eigvals_only=True)[0]
    return [float(lo - m) for m in margins]


@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("n_b,s_b", [(16, 32), (5, 70), (3, 130), (4, 256), (7, 1)])
def test_hermitian_sweeps_match_oracle(ss, prec, n_b, s_b):
    """The sweep blocks D_i factored as L D L^H without pivoting (the paper's
    no-pivoting Hermitian solver), updates on the lower triangle only: x, T and
    Sigma at the parity bar of the pivoted LU, at energies below the device's
    spectrum where every D_i is definite (the regime in which elimination
    without pivoting is stable; in band the blocks are indefinite)."""
    dev = synth.make_device(n_b, s_b, seed=120 + s_b)[0]
    Es = below_spectrum(dev, [0.5, 3.0])
    inj = [synth.make_injection(s_b, 3, seed=130 + i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj, precision=prec, hermitian_sweeps=1)
    assert np.all(np.asarray(r["st_T"]) == 0)
    for p in range(2):
        check_point(r, p, dev, Es[p], inj[p])


def test_hermitian_sweeps_with_partitions_and_lean_mode(ss):
    dev = synth.make_device(9, 48, seed=140, band=12, s_pert=0.02)[0]
    Es = below_spectrum(dev, [0.2, 1.5])
    inj = [synth.make_injection(48, 2, seed=141 + i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj, hermitian_sweeps=1, partitions=3)
    for p in range(2):
        check_point(r, p, dev, Es[p], inj[p])
    T, st = transmission_only(ss, [dev, dev], Es, hermitian_sweeps=1, precision=3)
    assert np.all(st == 0)
    for p in range(2):
        assert dense.rel_T_err(float(T[p]), float(r["T"][p])) < 1e-9


def test_hermitian_sweeps_report_pivot_growth(ss):
    """In band the blocks are indefinite and elimination without pivoting can
    blow up; where |L| exceeds 1e8 the point is reported singular rather than
    returned wrong.  (A device whose first diagonal block has a zero leading
    entry forces it.)"""
    dev = synth.make_device(3, 16, seed=151)[0]
    E = 0.2
    # A_11 entry (0, 0) = E S - H = 0: the first pivot of the block sweep's last block is zero
    dev.H_diag[0][0, 0] = E * dev.S_diag[0][0, 0]
    r = run_points(ss, [dev], [E], hermitian_sweeps=1)
    assert r["st_T"][0] == ss.SS_ERR_SINGULAR


def test_hermitian_sweeps_halve_the_factorisation_flops(ss):
    """The profiled algorithmic flops of the LU updates: with L D L^H the
    trailing update of the matrix part of each sweep block covers its lower
    triangle only, m (m + 1) / 2 instead of m^2 entries per panel (m rows below
    the panel), the right-hand sides and the back substitution unchanged."""
    dev = synth.make_device(6, 128, seed=150)[0]
    fl = {}
    for herm in (0, 1):
        h = ss.Handle(n_b_max=6, s_b_max=128, max_points=1, max_inj=1, profile=1, hermitian_sweeps=herm)
        try:
            h.set_device(0, dev)
            h.self_energy([0.2], [0])   # self-energies first: the next call profiles the sweeps only
            h.profile_reset()
            h.transmission([0.2], [0])
            fl[herm] = h.profile_read("zgemm_lu")[1]
        finally:
            h.close()
    nb, s_b, n_b = 16, 128, 6
    per_lu = sum(8.0 * nb * 0.5 * m * (m - 1) for m in (s_b - nb - k0 for k0 in range(0, s_b, nb)))
    expected = 2 * n_b * per_lu   # both sweep directions, every block
    assert abs((fl[0] - fl[1]) - expected) <= 1e-9 * fl[0], (fl, expected)


# ------------------------------------------------ whole-pipeline graph replay
@pytest.mark.parametrize("prec", [0, 3])
def test_repeated_batches_replay_graphs_bit_identically(ss, prec):
    """A second batch of the same shapes replays the sweep, boundary and
    refinement plans from CUDA graphs: the results equal eager launches bit for
    bit, and the host issues a few dozen launch calls instead of thousands."""
    dev = synth.make_device(6, 64, seed=160)[0]
    inj = [synth.make_injection(64, 2, seed=161 + i)[0] for i in range(2)]
    batches = [[0.1, -0.3], [0.45, -0.65], [0.2, 0.7]]
    out = {}
    for graphs in (0, 1):
        h = ss.Handle(n_b_max=6, s_b_max=64, max_points=2, max_inj=2, precision=prec, use_graphs=graphs)
        res, calls = [], []
        try:
            h.set_device(0, dev)
            for Es in batches:
                c0 = h.host_launch_count()
                xs, st, _ = h.solve(Es, [0, 0], inj)
                T, _, _, _ = h.transmission(Es, [0, 0])
                calls.append(h.host_launch_count() - c0)
                res.append((np.asarray(T).copy(), [np.asarray(x).copy() for x in xs], np.asarray(st)))
        finally:
            h.close()
        out[graphs] = (res, calls)
    for (Ta, xa, sa), (Tb, xb, sb) in zip(out[0][0], out[1][0]):
        assert np.all(sa == 0) and np.all(sb == 0)
        assert np.array_equal(Ta, Tb)
        assert all(np.array_equal(a, b) for a, b in zip(xa, xb))
    eager_calls, graph_calls = out[0][1], out[1][1]
    assert graph_calls[2] < 0.1 * eager_calls[2], (eager_calls, graph_calls)


# ------------------------------------------------- tournament pivoting panels
@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("n_b,s_b", [(16, 32), (5, 70), (3, 130), (2, 600)])
def test_tournament_pivoting_matches_oracle(ss, prec, n_b, s_b):
    """LU panels whose pivots come from a tournament over the cluster's CTAs
    (16-wide panels up to 512 rows, 8-wide up to 1024): x, T and Sigma at the
    parity bar of partial pivoting."""
    dev = synth.make_device(n_b, s_b, seed=170 + s_b)[0]
    Es = [0.3, -0.45]
    inj = [synth.make_injection(s_b, 3, seed=180 + i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj, precision=prec, tournament_pivoting=1)
    assert np.all(np.asarray(r["st_T"]) == 0)
    for p in range(2):
        check_point(r, p, dev, Es[p], inj[p])


def test_tournament_pivoting_reports_singular_and_nan(ss):
    dev = synth.make_device(3, 16, seed=16)[0]
    E = 0.4
    dev.H_diag[-1] = E * dev.S_diag[-1]   # A_nn = 0: the first pivot of the backward sweep is zero
    h = ss.Handle(n_b_max=3, s_b_max=16, max_points=1, max_inj=1, tournament_pivoting=1)
    try:
        h.set_device(0, dev)
        T, err, st, rc = h.transmission([E], [0])
    finally:
        h.close()
    assert st[0] == ss.SS_ERR_SINGULAR
    dev2 = synth.make_device(3, 16, seed=17)[0]
    dev2.H_diag[1][3, 3] = np.nan
    h = ss.Handle(n_b_max=3, s_b_max=16, max_points=1, max_inj=1, tournament_pivoting=1)
    try:
        h.set_device(0, dev2)
        T, err, st, rc = h.transmission([0.2], [0])
    finally:
        h.close()
    assert st[0] != ss.SS_OK

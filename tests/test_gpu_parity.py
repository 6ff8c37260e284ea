"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (FP64 path): relative error 1e-10 on T (|T - T_ref| /
max(1, |T_ref|)), on x (relative Frobenius) and on the self-energies
(relative Frobenius) -- or, where the problem itself is worse conditioned,
20 times the oracle's own sensitivity: the change of its result when H is
perturbed by one ulp (relative 2^-52 noise, two draws).  In band the doubling
at eta = 1e-10 amplifies rounding by up to ~1e6, so two correct FP64
implementations with different summation orders differ by that much.
Sizes span several 64-wide GEMM tiles, several 32-wide LU panels and ragged
tails.
"""
import numpy as np
import pytest

import synth
from oracle import channels, dense, leads

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def run_points(ss, devs, Es, inj=None, **cfg):
    """devs: list of synth.Device (one k_id each); Es: list of energies per point."""
    n_max = max(d.n_b for d in devs)
    s_max = max(d.s_b for d in devs)
    ninj = 1 if inj is None else max(a.shape[1] for a in inj)
    h = ss.Handle(n_b_max=n_max, s_b_max=s_max, max_points=cfg.pop("max_points", len(Es)),
                  max_inj=max(ninj, 1), **cfg)
    try:
        for k, d in enumerate(devs):
            h.set_device(k, d)
        kid = list(range(len(devs)))
        sL, sR, it, st_se, _ = h.self_energy(Es, kid)
        xs = None
        if inj is not None:
            xs, st_x, _ = h.solve(Es, kid, inj)
        T, err, st_T, _ = h.transmission(Es, kid)
        launches = h.launch_count()
    finally:
        h.close()
    return dict(sL=sL, sR=sR, iters=it, st_se=st_se, x=xs, T=T, st_T=st_T, launches=launches)


def noise_floor(dev, E, inj, ref):
    """Largest change of the oracle's outputs under one-ulp perturbations of H."""
    rng = np.random.default_rng(1234)
    out = dict(sL=0.0, sR=0.0, T=0.0, x=0.0)
    for _ in range(2):
        d2 = synth.Device(dev.H_diag * (1 + 2.0 ** -52 * rng.standard_normal(dev.H_diag.shape)),
                          dev.H_up * (1 + 2.0 ** -52 * rng.standard_normal(dev.H_up.shape)),
                          dev.S_diag, dev.S_up, lead_L=dev.lead_L, lead_R=dev.lead_R)
        r2 = dense.solve_point(d2, E, inj)
        out["sL"] = max(out["sL"], rel(r2["sigma_L"], ref["sigma_L"]))
        out["sR"] = max(out["sR"], rel(r2["sigma_R"], ref["sigma_R"]))
        out["T"] = max(out["T"], dense.rel_T_err(r2["T"], ref["T"]))
        if inj is not None:
            out["x"] = max(out["x"], rel(r2["x"], ref["x"]))
    return out


def check_point(r, p, dev, E, inj=None, tol=TOL):
    ref = dense.solve_point(dev, E, inj)
    nf = noise_floor(dev, E, inj, ref)
    t = {k: max(tol, 20.0 * v) for k, v in nf.items()}
    errs = dict(sL=rel(r["sL"][p], ref["sigma_L"]), sR=rel(r["sR"][p], ref["sigma_R"]),
                T=dense.rel_T_err(float(r["T"][p]), ref["T"]))
    if inj is not None:
        errs["x"] = rel(r["x"][p], ref["x"])
    for k, v in errs.items():
        assert v < t[k], (k, v, t[k], float(r["T"][p]), ref["T"])
    return ref


def test_small_config_point(ss):
    """n_b = 16, s_b = 32, one point E = 0.3 (the smallest workload)."""
    dev = synth.make_device(16, 32, seed=1)[0]
    inj = synth.make_injection(32, 4, seed=1)[0]
    r = run_points(ss, [dev], [0.3], [inj])
    assert r["st_T"][0] == 0 and r["st_se"][0] == 0
    ref = check_point(r, 0, dev, 0.3, inj)
    assert r["iters"][0, 0] == ref["info"]["iters_L"] or abs(r["iters"][0, 0] - ref["info"]["iters_L"]) <= 1
    assert r["launches"] > 0


@pytest.mark.parametrize("n_b,s_b", [(5, 70), (3, 130), (2, 33), (7, 1)])
def test_ragged_shapes(ss, n_b, s_b):
    dev = synth.make_device(n_b, s_b, seed=10 + s_b)[0]
    Es = [-0.4, 0.15]
    inj = [synth.make_injection(s_b, 3, seed=i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj)
    for p in range(2):
        check_point(r, p, dev, Es[p], inj[p])


def test_uneven_batch_in_one_call(ss):
    """Points with different (n_b, s_b) in the same launches (uneven batch)."""
    devs = [synth.make_device(6, 40, seed=2)[0], synth.make_device(3, 96, seed=3)[0],
            synth.make_device(9, 17, seed=4)[0]]
    Es = [0.2, -0.7, 0.55]
    inj = [synth.make_injection(d.s_b, 2, seed=5 + i)[0] for i, d in enumerate(devs)]
    r = run_points(ss, devs, Es, inj)
    for p, d in enumerate(devs):
        check_point(r, p, d, Es[p], inj[p])


def test_k_dependent_blocks(ss):
    devs = synth.make_device(4, 48, seed=6, k_points=synth.K_POINTS_4, w_scale=0.25)
    Es = [0.1, -0.3, 0.6, -0.9]
    r = run_points(ss, devs, Es)
    for p, d in enumerate(devs):
        check_point(r, p, d, Es[p])


def test_banded_blocks(ss):
    dev = synth.make_device(4, 100, seed=7, band=10, s_pert=0.02)[0]
    r = run_points(ss, [dev], [0.25])
    check_point(r, 0, dev, 0.25)


def test_explicit_leads_single_block(ss):
    """n_b = 1 with explicit leads (the smallest device)."""
    cell = synth.make_device(2, 12, seed=8)[0]
    lead = (cell.H_diag[0], cell.H_up[0], cell.S_diag[0], cell.S_up[0])
    dev = synth.Device(cell.H_diag[:1].copy(), np.zeros((0, 12, 12), np.complex128), cell.S_diag[:1].copy(),
                       np.zeros((0, 12, 12), np.complex128), lead_L=lead, lead_R=lead)
    inj = [synth.make_injection(12, 1, seed=3)[0]]
    r = run_points(ss, [dev], [0.05], inj)
    check_point(r, 0, dev, 0.05, inj[0])


def test_chain_closed_form_on_gpu(ss):
    """s_b = 1 chain: Sigma = t e^{ik}, T = 1 in band."""
    eps0, t = 0.2, -0.7
    dev = synth.Device(np.full((4, 1, 1), eps0, np.complex128), np.full((3, 1, 1), t, np.complex128),
                       np.ones((4, 1, 1), np.complex128), np.zeros((3, 1, 1), np.complex128))
    ks = [0.4, 1.3, 2.2]
    Es = [eps0 + 2 * t * np.cos(k) for k in ks]
    r = run_points(ss, [dev] * 3, Es)
    for p, k in enumerate(ks):
        assert abs(complex(r["sR"][p][0, 0]) - t * np.exp(1j * k)) < 1e-7
        assert abs(float(r["T"][p]) - 1.0) < 1e-8


def test_decoupled_wire_integer_T(ss):
    s, n, t = 24, 6, -0.8
    dev, eps = synth.decoupled_wire(s, n, t, seed=5)
    Es = []
    for E in np.linspace(-2.0, 2.0, 9):
        edges = np.concatenate([eps - 2 * abs(t), eps + 2 * abs(t)])
        if np.min(np.abs(E - edges)) > 0.05:
            Es.append(float(E))
    r = run_points(ss, [dev] * len(Es), Es)
    for p, E in enumerate(Es):
        expect = int(np.sum(np.abs(E - eps) < 2 * abs(t)))
        assert abs(float(r["T"][p]) - expect) < 1e-8


def test_periodic_wire_open_channels(ss):
    s, n = 16, 5
    dev, cell = synth.periodic_wire(s, n, seed=9)
    Es, ms = [], []
    for E in np.linspace(-3.0, 3.0, 13):
        lam = channels.bloch_factors(cell, E)
        dist = np.abs(np.abs(lam) - 1.0)
        if np.any((dist > 1e-8) & (dist < 5e-3)):
            continue
        Es.append(float(E))
        ms.append(channels.open_channels(cell, E)[0])
    r = run_points(ss, [dev] * len(Es), Es)
    for p in range(len(Es)):
        assert abs(float(r["T"][p]) - ms[p]) < 1e-6


def test_graph_replay_equals_eager_and_batching_is_exact(ss):
    dev = synth.make_device(5, 70, seed=12)[0]
    Es = [-0.2, 0.4]
    a = run_points(ss, [dev, dev], Es, use_graphs=1)
    b = run_points(ss, [dev, dev], Es, use_graphs=0)
    c0 = run_points(ss, [dev], [Es[0]])
    c1 = run_points(ss, [dev], [Es[1]])
    assert np.array_equal(np.asarray(a["T"]), np.asarray(b["T"]))
    assert float(a["T"][0]) == float(c0["T"][0]) and float(a["T"][1]) == float(c1["T"][0])
    assert np.array_equal(a["sL"][1], c1["sL"][0])


def test_chunking_beyond_max_points(ss):
    dev = synth.make_device(4, 40, seed=13)[0]
    Es = [-0.6, -0.1, 0.3, 0.8, 0.95]
    r = run_points(ss, [dev] * 5, Es, max_points=2)
    for p, E in enumerate(Es):
        assert dense.rel_T_err(float(r["T"][p]), dense.solve_point(dev, E)["T"]) < TOL


def test_device_pointer_mode_matches_host_mode(ss):
    import torch
    dev = synth.make_device(4, 40, seed=14)[0]
    inj = synth.make_injection(40, 3, seed=2)[0]
    E = 0.33
    host = run_points(ss, [dev], [E], [inj])
    h = ss.Handle(n_b_max=4, s_b_max=40, max_points=1, max_inj=3, device_ptrs=1,
                  stream=torch.cuda.current_stream().cuda_stream)
    try:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        h.set_hamiltonian(0, t(dev.H_diag), t(dev.H_up), t(dev.S_diag), t(dev.S_up))
        xs, st, _ = h.solve([E], [0], [t(inj)])
        T, err, st2, _ = h.transmission([E], [0])
        torch.cuda.synchronize()
    finally:
        h.close()
    assert np.array_equal(xs[0].cpu().numpy(), host["x"][0])
    assert float(T[0].item()) == float(host["T"][0])


# ------------------------------------------------------------ status paths
def test_decimation_cap_reports_not_converged(ss):
    dev = synth.make_device(3, 16, seed=15)[0]
    h = ss.Handle(n_b_max=3, s_b_max=16, max_points=1, max_inj=1, decim_max_iter=1)
    try:
        h.set_device(0, dev)
        sL, sR, it, st, rc = h.self_energy([0.1], [0])
    finally:
        h.close()
    assert rc == ss.SS_ERR_NOT_CONVERGED and st[0] == ss.SS_ERR_NOT_CONVERGED
    assert it[0, 0] == 1 and it[0, 1] == 1


def test_singular_block_reported(ss):
    dev = synth.make_device(3, 16, seed=16)[0]
    E = 0.4
    # A_nn = E S_nn - H_nn = 0: the first pivot of the backward sweep is zero
    dev.H_diag[-1] = E * dev.S_diag[-1]
    h = ss.Handle(n_b_max=3, s_b_max=16, max_points=1, max_inj=1)
    try:
        h.set_device(0, dev)
        T, err, st, rc = h.transmission([E], [0])
    finally:
        h.close()
    assert st[0] == ss.SS_ERR_SINGULAR and rc == ss.SS_ERR_SINGULAR


def test_nan_input_is_reported_not_hidden(ss):
    dev = synth.make_device(3, 16, seed=17)[0]
    dev.H_diag[1][3, 3] = np.nan
    h = ss.Handle(n_b_max=3, s_b_max=16, max_points=1, max_inj=1)
    try:
        h.set_device(0, dev)
        T, err, st, rc = h.transmission([0.2], [0])
    finally:
        h.close()
    assert st[0] != ss.SS_OK


def test_argument_and_state_errors(ss):
    h = ss.Handle(n_b_max=3, s_b_max=16, max_points=1, max_inj=1)
    try:
        with pytest.raises(ss.SSError) as e:
            h.transmission([0.2], [5])
        assert e.value.code == ss.SS_ERR_STATE
        dev = synth.make_device(4, 16, seed=1)[0]
        with pytest.raises(ss.SSError) as e:
            h.set_device(0, dev)      # n_b = 4 > n_b_max = 3
        assert e.value.code == ss.SS_ERR_ARG
    finally:
        h.close()


def test_workspace_too_large_is_oom(ss):
    with pytest.raises(ss.SSError) as e:
        ss.Handle(n_b_max=100000, s_b_max=4096, max_points=64)
    assert e.value.code == ss.SS_ERR_OOM


def test_caroli_transmission_entry_point(ss):
    """T from caller-provided Sigma_L, Sigma_R, G_1n (oracle values) on the device."""
    import torch
    pts = [(synth.make_device(4, 40, seed=20)[0], 0.3), (synth.make_device(4, 40, seed=21)[0], -0.5)]
    refs = [dense.solve_point(d, E) for d, E in pts]
    # the oracle's blocks may be Fortran-ordered views: pass dense row-major copies
    t = lambda key: torch.from_numpy(np.ascontiguousarray(np.stack([r[key] for r in refs]))).cuda()
    T = torch.zeros(2, dtype=torch.float64, device="cuda")
    ss.ss_caroli_transmission(t("sigma_L"), t("sigma_R"), t("G1n"), T)
    for p, r in enumerate(refs):
        assert dense.rel_T_err(float(T[p].item()), r["T"]) < 1e-12

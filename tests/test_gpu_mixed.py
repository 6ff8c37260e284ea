"""Mixed-precision pipeline (SS_MIXED_OZAKI) against the FP64 oracle.

Its products run on the tcgen05 tensor cores from BF16 digit slices with
exact FP32 accumulation, so it must meet the same bar as the FP64 path: 1e-10,
or 20 times the oracle's one-ulp sensitivity (see test_gpu_parity).  The
1e-8 bar on T for the mixed path is checked as well.
"""
import numpy as np
import pytest

import synth
from oracle import dense

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


@pytest.mark.parametrize("n_b,s_b", [(16, 32), (5, 70), (3, 130), (4, 256)])
def test_mixed_matches_oracle(ss, n_b, s_b):
    dev = synth.make_device(n_b, s_b, seed=30 + s_b)[0]
    Es = [0.3, -0.45]
    inj = [synth.make_injection(s_b, 3, seed=i)[0] for i in range(2)]
    r = run_points(ss, [dev, dev], Es, inj, precision=ss.SS_MIXED_OZAKI)
    for p in range(2):
        ref = check_point(r, p, dev, Es[p], inj[p])
        assert dense.rel_T_err(float(r["T"][p]), ref["T"]) <= 1e-8


def test_mixed_uneven_batch_and_k_points(ss):
    devs = synth.make_device(4, 96, seed=41, k_points=synth.K_POINTS_4[:2], w_scale=0.25) + \
        [synth.make_device(6, 40, seed=42)[0]]
    Es = [0.1, -0.3, 0.7]
    r = run_points(ss, devs, Es, precision=ss.SS_MIXED_OZAKI)
    for p, d in enumerate(devs):
        check_point(r, p, d, Es[p])


def test_mixed_agrees_with_fp64_path(ss):
    dev = synth.make_device(6, 128, seed=43, band=20, s_pert=0.02)[0]
    Es = [-0.8, 0.05, 0.6]
    a = run_points(ss, [dev] * 3, Es)
    b = run_points(ss, [dev] * 3, Es, precision=ss.SS_MIXED_OZAKI)
    for p in range(3):
        assert dense.rel_T_err(float(b["T"][p]), float(a["T"][p])) < 1e-9
        assert rel(b["sR"][p], a["sR"][p]) < 1e-8


def test_low_precision_modes_rejected_by_pipeline(ss):
    with pytest.raises(ss.SSError) as e:
        ss.Handle(n_b_max=4, s_b_max=32, max_points=1, precision=ss.SS_MIXED_BF16X3)
    assert e.value.code == ss.SS_ERR_ARG


def test_refinement_residual_reported_and_small(ss):
    """Mixed ss_solve refines x in FP64; ss_transmission reports its normwise
    backward error."""
    dev = synth.make_device(6, 96, seed=44)[0]
    Es = [0.25, -0.5]
    inj = [synth.make_injection(96, 4, seed=i)[0] for i in range(2)]
    h = ss.Handle(n_b_max=6, s_b_max=96, max_points=2, max_inj=4, precision=ss.SS_MIXED_OZAKI)
    try:
        h.set_device(0, dev)
        sL, sR, _, _, _ = h.self_energy(Es, [0, 0])
        xs, st, _ = h.solve(Es, [0, 0], inj)
        T, err, st2, _ = h.transmission(Es, [0, 0])
    finally:
        h.close()
    for p in range(2):
        # the residual of the refined x against the system with the GPU's own
        # self-energies (the oracle's differ by the doubling's conditioning)
        M = dense.system_matrix(dev, Es[p], sL[p], sR[p])
        b = dense.full_injection(inj[p], dev.n_b, dev.s_b)
        eta = dense.backward_error(M, xs[p], b)
        assert eta < 1e-14, eta
        # the estimate is max(backward error, |Im Tr| / max(1, T)); the first
        # carries the rounding of its own residual (about u sqrt(3 s_b)
        # relative to ||A - Sigma|| ||x||)
        assert 0.0 <= err[p] < 1e-12
        assert err[p] >= eta - 1e-14
        assert dense.residual(M, xs[p], b) < 1e-11
        check_point({"sL": sL, "sR": sR, "T": T, "x": xs}, p, dev, Es[p], inj[p])

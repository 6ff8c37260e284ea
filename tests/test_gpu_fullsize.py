"""The bench workload at full size, in the bench's launch configuration:
n_b = 64, s_b = 512, one batch of 8 (E,k) points (the first timed batch of
bench.py), CUDA graphs on, LU autotuned; mixed and FP64 paths.  The oracle's
recursive Green's function computes two of the points one by one; beyond
those samples the checks are properties that hold at any size: every point
converged (the refined x reached a backward error <= 1e-14, else its status
says so) and the two paths agree on T."""
import numpy as np
import pytest

import synth
from oracle import dense, rgf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def test_bench_batch_against_oracle_samples(ss, tmp_path):
    n_b, s_b, P, ninj = 64, 512, 8, 32
    devs = synth.make_device(n_b, s_b, seed=2, band=25, s_pert=0.02, k_points=synth.K_POINTS_4, w_scale=0.25)
    grid = synth.energy_grid(64)
    pts = [(float(e), k) for k in range(4) for e in grid][3 * P:4 * P]
    Es, Ks = [e for e, _ in pts], [k for _, k in pts]
    inj = synth.make_injection(s_b, ninj, seed=2, n_pts=P)
    T = {}
    for prec in (ss.SS_MIXED_OZAKI, ss.SS_FP64):
        h = ss.Handle(n_b_max=n_b, s_b_max=s_b, max_points=P, max_inj=ninj, precision=prec, use_graphs=1)
        try:
            for k, d in enumerate(devs):
                h.set_device(k, d)
            h.autotune(s_b, 2 * P, str(tmp_path / "tune.txt"))
            xs, st, _ = h.solve(Es, Ks, [inj[p] for p in range(P)])
            Tp, err, st2, _ = h.transmission(Es, Ks)
        finally:
            h.close()
        assert np.all(np.asarray(st) == 0) and np.all(np.asarray(st2) == 0), (prec, st, st2)
        assert all(np.all(np.isfinite(np.asarray(x))) for x in xs)
        T[prec] = np.asarray(Tp)
    # the mixed path's bar: T within 1e-8 of the FP64 path, and both within 1e-8 of the oracle
    rel = np.abs(T[ss.SS_MIXED_OZAKI] - T[ss.SS_FP64]) / np.maximum(1.0, np.abs(T[ss.SS_FP64]))
    assert np.max(rel) <= 1e-8, rel
    for p in (0, 2):
        E, k = pts[p]
        T_or = rgf.solve_point(devs[k], E)["T"]
        for prec in T:
            assert dense.rel_T_err(float(T[prec][p]), T_or) <= 1e-8, (prec, p, T[prec][p], T_or)

"""Autotuned LU settings: valid choice, on-disk cache round trip, and the
pipeline still matches the oracle with the tuned settings."""
import numpy as np
import pytest

import synth
from oracle import dense

from test_gpu_parity import check_point

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


@pytest.mark.parametrize("prec", [0, 3])
def test_autotune_cache_round_trip_and_parity(ss, tmp_path, prec):
    cache = tmp_path / "tune.txt"
    dev = synth.make_device(4, 96, seed=50)[0]
    h = ss.Handle(n_b_max=4, s_b_max=96, max_points=2, max_inj=2, precision=prec)
    try:
        nb, nbo, upd, ms = h.autotune(96, 4, cache)
        assert nb in (8, 16) and ms > 0
        assert (nbo, upd) in ([(0, 0)] if prec == 0 else
                              [(0, 0), (0, 2), (32, 2), (64, 2), (32, 3), (64, 3), (32, 4), (64, 4)])
        assert cache.read_text().split()[:6] == [str(prec), "96", "4", str(nb), str(nbo), str(upd)]
        assert h.autotune(96, 4, cache) == (nb, nbo, upd, pytest.approx(ms))
        h.set_device(0, dev)
        T, err, st, _ = h.transmission([0.2, -0.4], [0, 0])
    finally:
        h.close()
    for p, E in enumerate([0.2, -0.4]):
        assert dense.rel_T_err(float(T[p]), dense.solve_point(dev, E)["T"]) < 1e-9


# Forced LU blockings (a cache line is read back without timing): one- and
# two-level, outer widths that do and do not divide s_b = 300, exact
# products for the deep updates only or for all of them, and the two-level
# scheme with FP64 outer updates.
@pytest.mark.parametrize("prec,nb,nbo,upd", [(3, 16, 0, 2), (3, 8, 64, 2), (3, 16, 64, 2), (3, 16, 32, 2),
                                             (3, 16, 128, 2), (3, 8, 256, 2), (3, 16, 64, 3), (3, 8, 32, 3),
                                             (3, 16, 64, 0), (0, 16, 64, 0), (3, 16, 64, 4), (3, 8, 128, 4)])
def test_forced_blocking_parity(ss, tmp_path, prec, nb, nbo, upd):
    s_b, n_b = 300, 3
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{prec} {s_b} 4 {nb} {nbo} {upd} 1.0\n")
    dev = synth.make_device(n_b, s_b, seed=51)[0]
    inj = synth.make_injection(s_b, 3, seed=52, n_pts=2)
    Es = [0.15, -0.35]
    h = ss.Handle(n_b_max=n_b, s_b_max=s_b, max_points=2, max_inj=3, precision=prec)
    try:
        assert h.autotune(s_b, 4, cache) == (nb, nbo, upd, pytest.approx(1.0))
        h.set_device(0, dev)
        sL, sR, _, st0, _ = h.self_energy(Es, [0, 0])
        xs, st, _ = h.solve(Es, [0, 0], [inj[0], inj[1]])
        T, err, st2, _ = h.transmission(Es, [0, 0])
    finally:
        h.close()
    assert np.all(st0 == 0) and np.all(st == 0) and np.all(st2 == 0)
    for p, E in enumerate(Es):
        check_point({"sL": sL, "sR": sR, "T": T, "x": xs}, p, dev, E, inj[p])


def test_gemm_tile_tuning_is_recorded_and_changes_no_bit(ss, tmp_path):
    """ss_autotune also times the FP64 GEMM's tile shapes (square block products
    and the LU's rank-nb updates) and records them; every tile shape sums each
    output element in the same order, so the tuned plan gives bit-identical x
    and T to the heuristic tiles under the same LU blocking (the run with
    heuristic tiles reads back only the tuned blocking line, without timing)."""
    cache = tmp_path / "tune.txt"
    lu_only = tmp_path / "lu_only.txt"
    dev = synth.make_device(5, 128, seed=53)[0]
    inj = synth.make_injection(128, 2, seed=54, n_pts=2)
    Es = [0.25, -0.6]
    out = []
    for tuned in (True, False):
        h = ss.Handle(n_b_max=5, s_b_max=128, max_points=2, max_inj=2)
        try:
            if tuned:
                h.autotune(128, 4, cache)
                lu_only.write_text("".join(l + "\n" for l in cache.read_text().splitlines() if not l.startswith("G")))
            else:
                h.autotune(128, 4, lu_only)
            h.set_device(0, dev)
            xs, st, _ = h.solve(Es, [0, 0], [inj[0], inj[1]])
            T, _, st2, _ = h.transmission(Es, [0, 0])
        finally:
            h.close()
        out.append(([np.asarray(x).copy() for x in xs], np.asarray(T).copy()))
    assert "G" not in lu_only.read_text()
    g = [l.split() for l in cache.read_text().splitlines() if l.startswith("G")]
    assert len(g) == 1 and g[0][1:4] == ["0", "128", "4"]
    assert all(-1 <= int(v) <= 4 for v in g[0][4:6])  # -1: the heuristic was fastest
    assert np.array_equal(out[0][1], out[1][1])
    assert all(np.array_equal(a, b) for a, b in zip(out[0][0], out[1][0]))


# LU lookahead: the depth-nbo update of the columns right of the next outer
# block on a second stream, row exchanges of those columns deferred to the far
# phase.  Every element sees the same operations in the same order, so the
# results must not change by a single bit, eagerly or replayed from graphs.
@pytest.mark.parametrize("nb,nbo,upd", [(16, 64, 2), (8, 32, 4), (16, 128, 2), (16, 64, 0)])
def test_lu_lookahead_is_bit_identical(ss, tmp_path, nb, nbo, upd):
    s_b, n_b = 300, 3
    dev = synth.make_device(n_b, s_b, seed=71)[0]
    inj = synth.make_injection(s_b, 3, seed=72, n_pts=3)
    out = {}
    for la in (0, 1):
        cache = tmp_path / f"tune{la}.txt"
        cache.write_text(f"3 {s_b} 4 {nb} {nbo} {upd} 1.0\n")
        h = ss.Handle(n_b_max=n_b, s_b_max=s_b, max_points=3, max_inj=3, precision=3, lu_lookahead=la)
        try:
            assert h.autotune(s_b, 4, cache)[:3] == (nb, nbo, upd)
            h.set_device(0, dev)
            res = []
            for Es in ([0.15, -0.35, 0.5], [0.25, -0.45, 0.6]):  # the second batch replays the graphs
                sL, sR, _, st0, _ = h.self_energy(Es, [0, 0, 0])
                xs, st1, _ = h.solve(Es, [0, 0, 0], [inj[0], inj[1], inj[2]])
                T, _, st2, _ = h.transmission(Es, [0, 0, 0])
                assert np.all(np.asarray(st0) == 0) and np.all(np.asarray(st1) == 0) and np.all(np.asarray(st2) == 0)
                res.append(([np.asarray(a).copy() for a in sL] + [np.asarray(a).copy() for a in sR],
                            [np.asarray(x).copy() for x in xs], np.asarray(T).copy()))
        finally:
            h.close()
        out[la] = res
    for a, b in zip(out[0], out[1]):
        assert all(np.array_equal(u, v) for u, v in zip(a[0], b[0]))
        assert all(np.array_equal(u, v) for u, v in zip(a[1], b[1]))
        assert np.array_equal(a[2], b[2])
    # and the lookahead result is the oracle's
    for p, E in enumerate([0.15, -0.35, 0.5]):
        ref = dense.solve_point(dev, E, inj[p])
        assert dense.rel_T_err(float(out[1][0][2][p]), ref["T"]) < 1e-9

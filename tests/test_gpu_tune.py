"""Autotuned LU settings: valid choice, on-disk cache round trip, and the
pipeline still matches the oracle with the tuned settings."""
import numpy as np
import pytest

import synth
from oracle import dense

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
        nb, upd, ms = h.autotune(96, 4, cache)
        assert nb in (8, 16) and upd in ((0,) if prec == 0 else (0, 2)) and ms > 0
        assert cache.read_text().split()[:5] == [str(prec), "96", "4", str(nb), str(upd)]
        assert h.autotune(96, 4, cache) == (nb, upd, pytest.approx(ms))
        h.set_device(0, dev)
        T, err, st, _ = h.transmission([0.2, -0.4], [0, 0])
    finally:
        h.close()
    for p, E in enumerate([0.2, -0.4]):
        assert dense.rel_T_err(float(T[p]), dense.solve_point(dev, E)["T"]) < 1e-9

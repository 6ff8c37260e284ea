"""CPU checks of the warm-start feature map (independent of the oracle's)."""
import numpy as np

from oracle import mlp as omlp
from paper_1812_01396_gb300 import warm


def test_features_match_oracle_definition():
    rng = np.random.default_rng(0)
    E, k = rng.uniform(-1, 1, 50), rng.uniform(0, np.pi, 50)
    assert np.allclose(warm.features(E, k), omlp.features(E, k), rtol=1e-6, atol=1e-6)


def test_pack_targets_layout():
    g = np.arange(4).reshape(2, 2) + 1j * (10 + np.arange(4).reshape(2, 2))
    t = warm.pack_targets([g], 2.0)
    assert t.shape == (1, 8)
    assert np.allclose(t[0], [0, 2, 4, 6, 20, 22, 24, 26])
    assert np.allclose(omlp.unpack_g(t[0], 2, 2.0), g)

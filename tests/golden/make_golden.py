"""Writes tests/golden/small_case.json from the FP64 oracle only.

The small case (n_b = 16, s_b = 32, E = 0.3, seed 1, 4 injection columns,
seed 1) of the GPU parity tests and smoke(): the transmission, its imaginary
part, the Frobenius norms of the self-energies and of x, and a few entries.
The stored values guard the oracle against unintended changes; the oracle
itself is pinned by tests/test_oracle_pins.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import dense  # noqa: E402


def small_case():
    dev = synth.make_device(16, 32, seed=1)[0]
    inj = synth.make_injection(32, 4, seed=1)[0]
    r = dense.solve_point(dev, 0.3, inj)
    return {
        "case": "n_b=16, s_b=32, E=0.3, device seed 1, injection seed 1 (4 columns)",
        "T": float(r["T"]),
        "T_imag": float(r["T_imag"]),
        "T_RL": float(r["T_RL"]),
        "norm_sigma_L": float(np.linalg.norm(r["sigma_L"])),
        "norm_sigma_R": float(np.linalg.norm(r["sigma_R"])),
        "norm_x": float(np.linalg.norm(r["x"])),
        "sigma_L_00": [float(r["sigma_L"][0, 0].real), float(r["sigma_L"][0, 0].imag)],
        "x_00": [float(r["x"][0, 0].real), float(r["x"][0, 0].imag)],
        "doubling_iters": [int(r["info"]["iters_L"]), int(r["info"]["iters_R"])],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "small_case.json"), "w") as f:
        json.dump(small_case(), f, indent=1)
        f.write("\n")

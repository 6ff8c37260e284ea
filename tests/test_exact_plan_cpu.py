"""The exactness argument of the digit-sliced tensor-core GEMM, on the host:
the split the library plans for every inner size keeps each FP32 pass an
exact integer sum, covers every digit pair once, and covers 60 bits; and the
digit bounds the planner relies on hold for the digit recurrence."""
import numpy as np
import pytest

import paper_1812_01396_gb300 as ss

KS = sorted(set([1, 2, 3, 7, 16, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256, 300, 384,
                 511, 512, 513, 640, 768, 1000, 1024, 1536, 2047, 2048, 3000, 4096]))


@pytest.mark.parametrize("k", KS)
def test_plan_is_exact_and_complete(k):
    w, beta, S, passes = ss.exact_gemm_plan(k)
    assert w >= 2 * k and w % 64 == 0 and w < 2 * k + 64
    assert 3 <= beta <= 8            # |digit| <= 2^beta <= 256: exact in BF16 (8 significant bits)
    assert S * beta >= 60            # digits cover 60 bits below the row / column maximum
    assert len(passes) <= 32
    covered = {}
    for (d, t0, npairs) in passes:
        assert 0 <= d < S and npairs >= 1 and t0 + npairs - 1 <= d
        bound = 0
        for t in range(t0, t0 + npairs):
            u = d - t
            assert (t, u) not in covered
            covered[(t, u)] = True
            # leading digit <= 2^beta, later digits <= 2^(beta-1)
            bound += w * 2 ** (2 * beta - (t > 0) - (u > 0))
        assert bound <= 2 ** 24       # every partial sum is an integer FP32 holds exactly
    assert sorted(covered) == sorted((t, d - t) for d in range(S) for t in range(d + 1))


def _digits(x, e, beta, S):
    """The digit recurrence of the packing kernel, written from its definition:
    R = round(x 2^(62-e)) (|x| < 2^e), then for t = 0..S-1 with sh = 62 - beta (t+1):
    d_t = floor((R + 2^(sh-1)) / 2^sh), R -= d_t 2^sh, or d_t = R 2^(-sh) once sh <= 0."""
    R = int(round(x * 2.0 ** (62 - e)))
    out = []
    for t in range(S):
        sh = 62 - beta * (t + 1)
        if sh > 0:
            q = (R + (1 << (sh - 1))) >> sh
            R -= q << sh
        else:  # past the 62 fixed-point bits: the remainder, scaled up
            q = R << -sh
            R = 0
        out.append(q)
    return out, R


@pytest.mark.parametrize("beta", [3, 4, 5, 6, 7, 8])
def test_digit_bounds_and_reconstruction(beta):
    rng = np.random.default_rng(beta)
    S = (60 + beta - 1) // beta
    xs = list(rng.uniform(-1, 1, 2000)) + [1 - 2.0 ** -53, -(1 - 2.0 ** -53), 0.5, -0.5, 0.0, 2.0 ** -40]
    for x in xs:
        d, rem = _digits(float(x), 0, beta, S)
        assert abs(d[0]) <= 2 ** beta
        assert all(abs(q) <= 2 ** (beta - 1) for q in d[1:])
        recon = sum(q * 2.0 ** (-beta * (t + 1)) for t, q in enumerate(d))
        # what is left is below half a unit of the last digit (nothing once
        # the digits reach the 62 fixed-point bits)
        assert abs(rem) <= (2 ** (62 - beta * S - 1) if beta * S < 62 else 0)
        assert abs(recon - x) <= 2.0 ** (-min(beta * S, 62) - 1) + 2.0 ** -63

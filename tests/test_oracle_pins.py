"""Pins of the FP64 oracle against closed forms, brute force and identities.

None of these compares the oracle with itself: every expected value comes from
an independent construction (an analytic formula, a dense inverse assembled in
the test, or a physical invariant).
"""
import math

import numpy as np
import pytest

import synth
from oracle import alg1, channels, chol, dense, leads, mlp, rgf, warm


def chain_device(eps0, t, n_b=3):
    d = synth.Device(
        np.full((n_b, 1, 1), eps0, np.complex128), np.full((n_b - 1, 1, 1), t, np.complex128),
        np.ones((n_b, 1, 1), np.complex128), np.zeros((n_b - 1, 1, 1), np.complex128))
    return d


# ---------------------------------------------------------------- decimation
@pytest.mark.parametrize("k", [0.3, 1.0, 1.9, 2.8])
def test_chain_sigma_in_band(k):
    """1-D chain: Sigma = t e^{ik} at E = eps0 + 2 t cos k (t < 0), Im Sigma <= 0."""
    eps0, t = 0.2, -0.7
    E = eps0 + 2 * t * math.cos(k)
    sL, sR, info = leads.self_energies(chain_device(eps0, t), E)
    assert info["converged"]
    expect = t * np.exp(1j * k)
    assert abs(sR[0, 0] - expect) < 1e-7
    assert abs(sL[0, 0] - expect) < 1e-7
    assert sR[0, 0].imag <= 0 and sL[0, 0].imag <= 0


@pytest.mark.parametrize("E", [-2.5, 1.9, 3.0])
def test_chain_sigma_out_of_band(E):
    """Outside the band Sigma = t lambda with the decaying real root |lambda| < 1."""
    eps0, t = 0.2, -0.7
    sL, sR, _ = leads.self_energies(chain_device(eps0, t), E)
    dE = E - eps0
    roots = np.array([(dE + math.sqrt(dE * dE - 4 * t * t)) / 2, (dE - math.sqrt(dE * dE - 4 * t * t)) / 2])
    expect = roots[np.argmin(np.abs(roots))]
    assert abs(expect / t) < 1
    assert abs(sR[0, 0] - expect) < 1e-10
    assert abs(sR[0, 0].imag) < 1e-8


def _random_lead(s, seed):
    cell = synth.make_device(2, s, seed)[0]
    return (cell.H_diag[0], cell.H_up[0], cell.S_diag[0], cell.S_up[0])


def _chain_matrix(cell, z, ncell):
    """z S - H of a finite chain, assembled from the global Hermitian H and S."""
    H00, H01, S00, S01 = cell
    s = H00.shape[0]
    N = ncell * s
    H = np.zeros((N, N), np.complex128)
    S = np.zeros((N, N), np.complex128)
    for q in range(ncell):
        H[q * s:(q + 1) * s, q * s:(q + 1) * s] = H00
        S[q * s:(q + 1) * s, q * s:(q + 1) * s] = S00
    for q in range(ncell - 1):
        H[q * s:(q + 1) * s, (q + 1) * s:(q + 2) * s] = H01
        S[q * s:(q + 1) * s, (q + 1) * s:(q + 2) * s] = S01
        H[(q + 1) * s:(q + 2) * s, q * s:(q + 1) * s] = H01.conj().T
        S[(q + 1) * s:(q + 2) * s, q * s:(q + 1) * s] = S01.conj().T
    return z * S - H


@pytest.mark.parametrize("seed", [11, 12])
def test_doubling_iterates_equal_finite_chain_inverse(seed):
    """After j doublings: es_R^-1 = [M_{0..2^j-1}^-1]_{00}, es_L^-1 = last block,
    e^-1 = centre block of the (2^{j+1}-1)-cell chain."""
    s = 4
    cell = _random_lead(s, seed)
    z = 0.37 + 0.05j
    D, U, L = leads.lead_matrices(cell, z)
    r = leads.sancho_rubio(D, U, L, tol=0.0, max_iter=5, history=True)
    for j, (esR, esL, e) in enumerate(r["hist"], start=1):
        n = 2 ** j
        Minv = np.linalg.inv(_chain_matrix(cell, z, n))
        assert np.allclose(np.linalg.inv(esR), Minv[:s, :s], rtol=1e-9, atol=1e-11)
        assert np.allclose(np.linalg.inv(esL), Minv[-s:, -s:], rtol=1e-9, atol=1e-11)
        m = 2 ** (j + 1) - 1
        c = 2 ** j - 1
        Minv = np.linalg.inv(_chain_matrix(cell, z, m))
        assert np.allclose(np.linalg.inv(e), Minv[c * s:(c + 1) * s, c * s:(c + 1) * s],
                           rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("E", [-0.6, 0.1, 0.8])
def test_surface_gf_dyson_and_spectral_psd(E):
    s = 6
    cell = _random_lead(s, 21)
    z = E + 1j * leads.DEFAULT_ETA
    D, U, L = leads.lead_matrices(cell, z)
    for side in ("R", "L"):
        g, it, conv = leads.surface_gf(cell, z, side)
        assert conv and it < 100
        assert warm.dyson_residual(g, D, U, L, side) < 1e-9
        A = 1j * (g - g.conj().T)
        w = np.linalg.eigvalsh((A + A.conj().T) / 2)
        assert w.min() >= -1e-9 * max(1.0, w.max())


def test_decimation_cap_reports_not_converged():
    cell = _random_lead(4, 3)
    D, U, L = leads.lead_matrices(cell, 0.1 + 1e-10j)
    r = leads.sancho_rubio(D, U, L, max_iter=1)
    assert r["iters"] == 1 and not r["converged"]


# ----------------------------------------------------------- transmission
def test_decoupled_wire_integer_transmission():
    s, n, t = 6, 5, -0.8
    dev, eps = synth.decoupled_wire(s, n, t, seed=5)
    for E in np.linspace(-2.0, 2.0, 17):
        edges = np.concatenate([eps - 2 * abs(t), eps + 2 * abs(t)])
        if np.min(np.abs(E - edges)) < 0.05:
            continue
        expect = int(np.sum(np.abs(E - eps) < 2 * abs(t)))
        r = dense.solve_point(dev, E)
        assert abs(r["T"] - expect) < 1e-8, (E, r["T"], expect)


def test_periodic_wire_transmission_equals_open_channels():
    s, n = 4, 4
    dev, cell = synth.periodic_wire(s, n, seed=9)
    checked = 0
    for E in np.linspace(-3.0, 3.0, 25):
        lam = channels.bloch_factors(cell, E)
        dist = np.abs(np.abs(lam) - 1.0)
        if np.any((dist > 1e-8) & (dist < 5e-3)):
            continue          # too close to a band edge
        m, _ = channels.open_channels(cell, E)
        r = dense.solve_point(dev, E)
        assert abs(r["T"] - m) < 1e-6, (E, r["T"], m)
        checked += 1
    assert checked >= 10


# -------------------------------------------------------------- Algorithm 1
def test_alg1_columns_equal_dense_inverse():
    dev = synth.make_device(5, 4, seed=1)[0]
    E = 0.3
    Ainv = np.linalg.inv(dense.assemble_A(dev, E))
    Qf = alg1.first_block_column(dev, E)
    Ql = alg1.last_block_column(dev, E)
    s = 4
    for i in range(5):
        assert np.allclose(Qf[i], Ainv[i * s:(i + 1) * s, :s], rtol=1e-12, atol=1e-13)
        assert np.allclose(Ql[i], Ainv[i * s:(i + 1) * s, -s:], rtol=1e-12, atol=1e-13)


def test_smw_steps_equal_dense_open_system():
    dev = synth.make_device(6, 3, seed=2)[0]
    E = -0.2
    inj = synth.make_injection(3, 2, seed=4)[0]
    r = dense.solve_point(dev, E, inj)
    x, R, g, Gb = alg1.smw_solve(dev, E, r["sigma_L"], r["sigma_R"], inj)
    assert np.allclose(x, r["x"], rtol=1e-11, atol=1e-12)
    s = 3
    Minv = np.linalg.inv(r["M"])
    corners = np.block([[Minv[:s, :s], Minv[:s, -s:]], [Minv[-s:, :s], Minv[-s:, -s:]]])
    assert np.allclose(Gb, corners, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("E", [-0.5, 0.3])
def test_open_system_invariants(E):
    dev = synth.make_device(6, 5, seed=3)[0]
    r = dense.solve_point(dev, E)
    s = 5
    gl, gr = leads.gamma(r["sigma_L"]), leads.gamma(r["sigma_R"])
    for G in (gl, gr):
        assert np.allclose(G, G.conj().T, atol=1e-13)
        w = np.linalg.eigvalsh(G)
        assert w.min() >= -1e-10 * w.max()
    # Ward identity on the corners
    G11, G1n, Gnn, Gn1 = r["G11"], r["G1n"], r["Gnn"], r["Gn1"]
    lhs = 1j * (G11 - G11.conj().T)
    rhs = G11 @ gl @ G11.conj().T + G1n @ gr @ G1n.conj().T
    assert np.allclose(lhs, rhs, rtol=1e-8, atol=1e-8 * np.abs(lhs).max())
    lhs = 1j * (Gnn - Gnn.conj().T)
    rhs = Gn1 @ gl @ Gn1.conj().T + Gnn @ gr @ Gnn.conj().T
    assert np.allclose(lhs, rhs, rtol=1e-8, atol=1e-8 * np.abs(lhs).max())
    # reciprocity, reality, bounds
    assert abs(r["T"] - r["T_RL"]) <= 1e-10 * max(1, r["T"])
    assert abs(r["T_imag"]) <= 1e-10 * max(1, r["T"])
    left, right = leads.lead_cells(dev)
    mL, _ = channels.open_channels(left, E)
    mR, _ = channels.open_channels(right, E)
    assert -1e-10 <= r["T"] <= min(mL, mR) + 1e-8


def test_injection_current_conservation_and_residual():
    dev = synth.make_device(7, 4, seed=8)[0]
    E = 0.2
    r0 = dense.solve_point(dev, E)
    # keep every positive pivot: then Gamma_R = V V^H to rounding
    V, _ = chol.pivoted_cholesky(leads.gamma(r0["sigma_R"]), rtol=1e-15)
    inj = np.vstack([np.zeros((4, V.shape[1])), V])
    r = dense.solve_point(dev, E, inj)
    x = r["x"]
    assert dense.residual(r["M"], x, r["inj_full"]) < 1e-13
    J = dense.bond_currents(dev, E, x)
    assert np.allclose(J, J[0], rtol=1e-10, atol=1e-12)
    x1 = x[:4]
    T_inj = np.real(np.trace(x1.conj().T @ leads.gamma(r["sigma_L"]) @ x1))
    assert abs(T_inj - r["T"]) < 1e-10 * max(1, r["T"])
    # the current carried equals the transmission (one unit per channel)
    assert abs(abs(J[0]) - r["T"]) < 1e-8 * max(1, r["T"])
    # dropping the eta-sized pivots (default rtol) changes T far below 1e-8
    V2, _ = chol.pivoted_cholesky(leads.gamma(r0["sigma_R"]))
    x2 = dense.solve_point(dev, E, np.vstack([np.zeros((4, V2.shape[1])), V2]))["x"][:4]
    T2 = np.real(np.trace(x2.conj().T @ leads.gamma(r["sigma_L"]) @ x2))
    assert abs(T2 - r["T"]) < 1e-8


def test_rgf_matches_dense():
    dev = synth.make_device(6, 5, seed=6)[0]
    inj = synth.make_injection(5, 3, seed=1)[0]
    a = dense.solve_point(dev, 0.25, inj)
    b = rgf.solve_point(dev, 0.25, inj)
    for key in ("G11", "G1n", "Gn1", "Gnn", "x"):
        assert np.allclose(a[key], b[key], rtol=1e-10, atol=1e-12), key
    assert abs(a["T"] - b["T"]) < 1e-11


def test_pivoted_cholesky_recovers_low_rank():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    G = B @ B.conj().T
    V, piv = chol.pivoted_cholesky(G)
    assert V.shape[1] == 3
    assert np.allclose(V @ V.conj().T, G, atol=1e-12)
    assert len(set(piv)) == 3


# --------------------------------------------------------------------- MLP
def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = mlp.init_params(6, width=8, seed=3)
    x = mlp.features(rng.uniform(-1, 1, 4), rng.uniform(0, 3, 4))
    t = rng.standard_normal((4, 6))
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t)
    h = 1e-6
    for pi in range(6):
        p = params[pi]
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, min(5, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(params, x)[0], t)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(params, x)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[pi].reshape(-1)[idx]) <= 1e-6 * max(1e-3, abs(fd)), (pi, idx)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected step is lr * g / (|g| + eps)."""
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.3, -0.5])]
    m = [np.zeros(2)]
    v = [np.zeros(2)]
    for t in range(1, 4):
        prev = p[0].copy()
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=0.01)
        step = prev - p[0]
        assert np.allclose(step, 0.01 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-12)


def test_backward_error_is_the_smallest_perturbation():
    """Rigal-Gaches: the perturbation dM = -t r x^H / ||x||^2 * a, db = t r * c
    with a = ||M|| ||x|| / (||M|| ||x|| + ||b||), c = ||b|| / (...) makes x an
    exact solution and has ||dM|| = eta ||M||, ||db|| = eta ||b||."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))
    x = rng.standard_normal((7, 2)) + 1j * rng.standard_normal((7, 2))
    b = rng.standard_normal((7, 2)) + 1j * rng.standard_normal((7, 2))
    eta = dense.backward_error(M, x, b)
    nM, nx, nb = np.linalg.norm(M), np.linalg.norm(x), np.linalg.norm(b)
    r = b - M @ x
    # x is a matrix: use the minimum-norm dM with dM x = a r (Frobenius)
    a, c = nM * nx / (nM * nx + nb), nb / (nM * nx + nb)
    dM = a * r @ np.linalg.pinv(x)
    db = -c * r
    assert np.allclose((M + dM) @ x, b + db, atol=1e-12)
    assert np.linalg.norm(db) == pytest.approx(eta * nb, rel=1e-12)
    # for a single right-hand side the minimum-norm dM is rank one with norm eta ||M||
    x1, b1 = x[:, :1], b[:, :1]
    e1 = dense.backward_error(M, x1, b1)
    r1 = b1 - M @ x1
    n1 = np.linalg.norm(M) * np.linalg.norm(x1) + np.linalg.norm(b1)
    dM1 = (np.linalg.norm(M) * np.linalg.norm(x1) / n1) * r1 @ x1.conj().T / np.linalg.norm(x1) ** 2
    assert np.allclose((M + dM1) @ x1, b1 - (np.linalg.norm(b1) / n1) * r1, atol=1e-12)
    assert np.linalg.norm(dM1) == pytest.approx(e1 * np.linalg.norm(M), rel=1e-12)
    # closed form: M = I, b = 0 -> ||x|| / (sqrt(N) ||x||)
    assert dense.backward_error(np.eye(9), np.ones((9, 1)), np.zeros((9, 1))) == pytest.approx(1 / 3, rel=1e-15)
    # an exact solution has zero backward error
    M2 = np.diag([1.0, 2.0, 4.0])
    assert dense.backward_error(M2, np.array([[1.0], [0.5], [0.25]]), np.ones((3, 1))) == 0.0


def test_oracle_reproduces_golden_small_case():
    """The small case's stored oracle outputs (written by
    tests/golden/make_golden.py from the oracle only) are reproduced: a guard
    against unintended changes of the oracle's arithmetic.  The tolerance
    (1e-8) leaves room for another BLAS: the lead doubling at eta = 1e-10
    amplifies rounding differences by up to about 1e6."""
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_case.json")
    gold = json.load(open(here))
    dev = synth.make_device(16, 32, seed=1)[0]
    inj = synth.make_injection(32, 4, seed=1)[0]
    r = dense.solve_point(dev, 0.3, inj)
    assert r["T"] == pytest.approx(gold["T"], rel=1e-8)
    assert r["T_RL"] == pytest.approx(gold["T_RL"], rel=1e-8)
    assert abs(r["T_imag"]) < 1e-12
    assert np.linalg.norm(r["sigma_L"]) == pytest.approx(gold["norm_sigma_L"], rel=1e-8)
    assert np.linalg.norm(r["sigma_R"]) == pytest.approx(gold["norm_sigma_R"], rel=1e-8)
    assert np.linalg.norm(r["x"]) == pytest.approx(gold["norm_x"], rel=1e-8)
    assert complex(*gold["sigma_L_00"]) == pytest.approx(complex(r["sigma_L"][0, 0]), rel=1e-7)
    assert complex(*gold["x_00"]) == pytest.approx(complex(r["x"][0, 0]), rel=1e-7)
    assert [r["info"]["iters_L"], r["info"]["iters_R"]] == gold["doubling_iters"]


# ------------------------------------------------------------ MLP forward
def test_mlp_forward_hand_computed_network():
    """A 3 -> 2 -> 2 -> 3 network whose pre-activations are +-ln 3 and 0, where
    SiLU is known in closed form: sigma(ln 3) = 3/4, so SiLU(ln 3) = 0.75 ln 3,
    SiLU(-ln 3) = -0.25 ln 3, SiLU(0) = 0.  The square middle layer is not
    symmetric, so W in place of W^T changes the result; the first and last
    layers are not square, so a transposed layout fails outright."""
    L = math.log(3.0)
    W1 = np.array([[L, 0.0, 0.0], [0.0, 0.0, L]])
    b1 = np.zeros(2)
    W2 = np.array([[1.0, -1.0], [1.0, 3.0]])
    b2 = np.zeros(2)
    W3 = np.array([[2.0, 5.0], [0.0, 1.0], [-4.0, 7.0]])
    b3 = np.array([0.5, 0.0, 1.0])
    x = np.array([[1.0, 2.0, -1.0]])
    y, cache = mlp.forward([W1, b1, W2, b2, W3, b3], x)
    _, h1, a1, h2, a2 = cache
    assert np.allclose(h1, [[L, -L]], rtol=0, atol=1e-15)
    assert np.allclose(a1, [[0.75 * L, -0.25 * L]], rtol=0, atol=1e-15)
    assert np.allclose(h2, [[L, 0.0]], rtol=0, atol=1e-15)
    assert np.allclose(a2, [[0.75 * L, 0.0]], rtol=0, atol=1e-15)
    assert np.allclose(y, [[1.5 * L + 0.5, 0.0, -3.0 * L + 1.0]], rtol=0, atol=1e-14)


def test_mlp_silu_identities():
    """SiLU(0) = 0, SiLU(-x) = SiLU(x) - x, SiLU(x) -> x for large x."""
    xs = np.array([0.3, 1.7, 4.0, 12.0])
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.silu(-xs), mlp.silu(xs) - xs, rtol=0, atol=1e-15)
    assert abs(mlp.silu(np.array([40.0]))[0] - 40.0) < 1e-15


def test_mlp_features_at_known_angles():
    """Feature order (E, cos k, sin k, sin(m pi E), cos(m pi E), m = 1..8) at
    E = 1/2, k = pi/2, where every entry is 0 or +-1."""
    f = mlp.features([0.5], [math.pi / 2])[0]
    assert f.shape == (19,)
    assert f[0] == 0.5
    assert abs(f[1]) < 1e-15 and abs(f[2] - 1.0) < 1e-15
    sin_m = [1, 0, -1, 0, 1, 0, -1, 0]
    cos_m = [0, -1, 0, 1, 0, -1, 0, 1]
    for m in range(8):
        assert abs(f[3 + 2 * m] - sin_m[m]) < 1e-14
        assert abs(f[4 + 2 * m] - cos_m[m]) < 1e-14


# ------------------------------------------------------ seeded fixed point
@pytest.mark.parametrize("E", [-2.5, 3.0])
def test_fixed_point_converges_to_chain_closed_form_out_of_band(E):
    """s = 1 chain, out of band: the map g <- (D - U g L)^-1 contracts by
    |lambda|^2 < 1 and its fixed point is g_R = Sigma / t^2 with Sigma = t lambda,
    lambda the decaying root (the closed form of the decimation pins)."""
    eps0, t = 0.2, -0.7
    z = E + 1j * leads.DEFAULT_ETA
    D = np.array([[z - eps0]])
    U = np.array([[-t + 0j]])
    L = np.array([[-t + 0j]])
    # Sigma^2 - (z - eps0) Sigma + t^2 = 0 at the complex z of the map
    dz = z - eps0
    sq = np.sqrt(complex(dz * dz - 4 * t * t))
    roots = np.array([(dz + sq) / 2, (dz - sq) / 2])
    sigma = roots[np.argmin(np.abs(roots))]
    assert abs(sigma / t) < 1
    for side in ("R", "L"):
        g = warm.fixed_point(np.zeros((1, 1)), D, U, L, side=side, iters=60)
        assert abs(g[0, 0] - sigma / t ** 2) < 1e-13
        assert warm.dyson_residual(g, D, U, L, side) < 1e-14


@pytest.mark.parametrize("E", [-0.4, 0.7])
def test_fixed_point_keeps_the_doubling_result(E):
    """For a random lead (U != L^T, so the order U g L versus L g U matters) the
    surface Green's function of the independent doubling is a fixed point of the
    map of each side: one step moves it only by rounding."""
    cell = _random_lead(6, 31)
    z = E + 1j * leads.DEFAULT_ETA
    D, U, Lm = leads.lead_matrices(cell, z)
    for side in ("R", "L"):
        g, _, conv = leads.surface_gf(cell, z, side)
        assert conv
        g1 = warm.fixed_point(g, D, U, Lm, side=side, iters=1)
        assert np.linalg.norm(g1 - g) / np.linalg.norm(g) < 1e-9
        other = "L" if side == "R" else "R"
        g_wrong = warm.fixed_point(g, D, U, Lm, side=other, iters=1)
        assert np.linalg.norm(g_wrong - g) / np.linalg.norm(g) > 1e-3


# ----------------------------------------------------------- open channels
def test_open_channels_of_decoupled_wire_closed_form():
    """Decoupled wire: chain j carries one right-moving mode iff |E - eps_j| < 2|t|."""
    s, t = 10, -0.8
    dev, eps = synth.decoupled_wire(s, 3, t, seed=4)
    cell = (dev.H_diag[0], dev.H_up[0], dev.S_diag[0], dev.S_up[0])
    for E in (-2.1, -0.9, 0.05, 1.3, 2.4):
        edges = np.concatenate([eps - 2 * abs(t), eps + 2 * abs(t)])
        if np.min(np.abs(E - edges)) < 0.02:
            continue
        expect = int(np.sum(np.abs(E - eps) < 2 * abs(t)))
        m, n_unit = channels.open_channels(cell, E)
        assert m == expect and n_unit == 2 * expect


# ------------------------------------------------------- density of states
@pytest.mark.parametrize("k", [0.4, 1.3, 2.5])
def test_ldos_of_perfect_chain_closed_form(k):
    """A perfect 1-D chain (device cells equal to the lead cells): every site
    carries the bulk density of states 1 / (pi sqrt(4 t^2 - (E - eps0)^2)) in band."""
    eps0, t = 0.2, -0.7
    E = eps0 + 2 * t * math.cos(k)
    rho = dense.ldos(chain_device(eps0, t, n_b=5), E)
    expect = 1.0 / (math.pi * math.sqrt(4 * t * t - (E - eps0) ** 2))
    assert np.allclose(rho, expect, rtol=1e-8, atol=0)


def test_ldos_of_decoupled_wire_closed_form():
    """Decoupled wire: the trace is basis independent, so each cell's LDOS is the
    sum of the 1-D bulk densities of the chains whose band holds E (zero in gaps)."""
    s, t = 8, -0.8
    dev, eps = synth.decoupled_wire(s, 4, t, seed=6)
    for E in (-1.9, -0.3, 0.6, 2.2):
        edges = np.concatenate([eps - 2 * abs(t), eps + 2 * abs(t)])
        if np.min(np.abs(E - edges)) < 0.05:
            continue
        inb = np.abs(E - eps) < 2 * abs(t)
        expect = float(np.sum(1.0 / (np.pi * np.sqrt(4 * t * t - (E - eps[inb]) ** 2))))
        rho = dense.ldos(dev, E)
        assert np.allclose(rho, expect, rtol=1e-7, atol=1e-9), (E, rho, expect)


# ------------------------------------------------------ modes (FEAST route)
@pytest.mark.parametrize("s,seed", [(6, 31), (12, 5)])
@pytest.mark.parametrize("E", [-0.4, 0.7, 3.0])
def test_mode_self_energies_equal_decimation(s, seed, E):
    """Sigma from the lead's Bloch modes (all of them inside the annulus) is the
    same quantity as the decimation's, by an independent route: a generalized
    eigensolver on the companion pencil instead of the doubling."""
    from oracle import feast
    dev = synth.make_device(3, s, seed)[0]
    sL, sR, _ = leads.self_energies(dev, E)
    fL, fR, info = feast.self_energies(dev, E)
    assert info["modes_L"] == s and info["modes_R"] == s
    assert np.linalg.norm(fL - sL) / np.linalg.norm(sL) < 1e-10
    assert np.linalg.norm(fR - sR) / np.linalg.norm(sR) < 1e-10


@pytest.mark.parametrize("k", [0.4, 1.3, 2.5])
def test_mode_self_energy_of_chain(k):
    """s = 1 chain: the right-going mode is lambda = e^{ik}, Sigma = t e^{ik}."""
    from oracle import feast
    eps0, t = 0.2, -0.7
    E = eps0 + 2 * t * math.cos(k)
    sL, sR, info = feast.self_energies(chain_device(eps0, t), E)
    assert abs(sR[0, 0] - t * np.exp(1j * k)) < 1e-7 and abs(sL[0, 0] - t * np.exp(1j * k)) < 1e-7


def test_mode_counts_and_annulus():
    """Each direction has s modes; the unimodular ones number twice the open
    channels; shrinking the annulus drops only fast-decaying modes."""
    from oracle import feast
    s, t = 10, -0.8
    dev, eps = synth.decoupled_wire(s, 3, t, seed=4)
    cell = (dev.H_diag[0], dev.H_up[0], dev.S_diag[0], dev.S_up[0])
    E = 0.05
    lam, u = feast.lead_modes(cell, E + 1j * leads.DEFAULT_ETA)
    assert np.sum(np.abs(lam) < 1) == s and np.sum(np.abs(lam) > 1) == s
    assert np.sum(np.abs(np.abs(lam) - 1) < 1e-6) == 2 * channels.open_channels(cell, E)[0]
    g_all, m_all = feast.surface_gf(cell, E + 1j * leads.DEFAULT_ETA, "R")
    g_cut, m_cut = feast.surface_gf(cell, E + 1j * leads.DEFAULT_ETA, "R", R=4.0)
    assert m_all == s and m_cut == int(np.sum((np.abs(lam) < 1) & (np.abs(lam) > 0.25)))

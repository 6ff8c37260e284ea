"""Learned warm start: the network kernels against the FP64 oracle MLP, and
the warm-started surface Green's function against plain doubling.

Bars: forward and gradients within 1e-2 (relative, per tensor) of the FP64
oracle run with the same BF16-rounded weights and inputs (the kernels keep
activations in BF16 and accumulate in FP32).  Every warm-start result equals
the plain doubling to the conditioning bar: accepted seeds satisfy the FP64
Dyson residual test, rejected ones fall back to the doubling itself.
"""
import time

import numpy as np
import pytest

import synth
from oracle import dense
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def bf16(a):
    """Round float32 to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("width,n_out,batch,tc", [
    (48, 32, 12, True),      # one tile, ragged in every dimension
    (48, 32, 12, False),     # the SIMT kernel on the same case
    (136, 264, 200, True),   # 2 x 3 output tiles, ragged M / N / K tails, K = 19 through a padded row stride
    (36, 18, 9, False),      # widths that are not multiples of 8 run on the SIMT kernel only
])
def test_mlp_forward_and_gradients_match_oracle(ss, width, n_out, batch, tc):
    import torch
    from paper_1812_01396_gb300 import warm
    net = ss.MLP(19, width, n_out, batch + 3, seed=3)
    if (width % 8 or n_out % 8) and tc:
        pytest.skip("tensor cores need multiples of 8")
    if width % 8 or n_out % 8:
        with pytest.raises(ss.SSError):
            net.use_tensor_cores(True)
    net.use_tensor_cores(tc)
    params = [p.astype(np.float32) for p in omlp.init_params(n_out, width=width, seed=4)]
    params = [p + 0.05 * np.float32(i % 2) for i, p in enumerate(params)]   # non-zero biases
    net.set_params(params)
    rng = np.random.default_rng(2)
    E, k = rng.uniform(-1, 1, batch), rng.uniform(0, np.pi, batch)
    x = warm.features(E, k)
    t = rng.standard_normal((batch, n_out)).astype(np.float32)
    tx, tt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(tx).cpu().numpy()
    net.train_step(tx, tt, 0.0)
    grads = net.get_grads()
    op = [bf16(p) if i % 2 == 0 else p.astype(np.float64) for i, p in enumerate(params)]
    yo, cache = omlp.forward(op, bf16(x))
    go = omlp.backward(op, cache, yo, t.astype(np.float64))
    assert rel(y, yo) < 1e-2
    for i in range(6):
        assert rel(grads[i], go[i]) < 1e-2, (i, rel(grads[i], go[i]))
    net.close()


def test_mlp_tensor_cores_match_simt_and_step_time(ss, capsys):
    """The warm-start network at its workload size (width 512, n_out 2 * 128^2,
    batch 256): tensor-core and SIMT GEMMs give the same outputs and gradients
    to BF16 rounding (both round the same operands, both accumulate in FP32);
    reports the time of one training step on each."""
    import torch
    from paper_1812_01396_gb300 import warm
    W, O, B = 512, 2 * 128 * 128, 256
    rng = np.random.default_rng(5)
    x = torch.from_numpy(warm.features(rng.uniform(-1, 1, B), rng.uniform(0, np.pi, B))).cuda()
    t = torch.from_numpy(rng.standard_normal((B, O)).astype(np.float32)).cuda()
    out = {}
    for tc in (True, False):
        net = ss.MLP(19, W, O, B, seed=8)
        net.use_tensor_cores(tc)
        y = net.forward(x).cpu().numpy()
        loss = net.train_step(x, t, 0.0)
        g = net.get_grads()
        for _ in range(3):
            net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        t0 = time.time()
        for _ in range(20):
            net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        out[tc] = dict(y=y, loss=loss, g=g, ms=(time.time() - t0) / 20 * 1e3)
        net.close()
    assert rel(out[True]["y"], out[False]["y"]) < 1e-2
    assert abs(out[True]["loss"] - out[False]["loss"]) < 1e-2 * out[False]["loss"]
    for i in range(6):
        assert rel(out[True]["g"][i], out[False]["g"][i]) < 2e-2, i
    with capsys.disabled():
        print("\nMLP training step (19 -> 512 -> 512 -> 32768, batch 256): tensor cores %.3f ms, SIMT %.3f ms"
              % (out[True]["ms"], out[False]["ms"]))


def test_mlp_training_reduces_loss(ss):
    import torch
    from paper_1812_01396_gb300 import warm
    net = ss.MLP(19, 64, 16, 64, seed=1)
    rng = np.random.default_rng(0)
    E = rng.uniform(-1, 1, 64)
    x = torch.from_numpy(warm.features(E, np.zeros(64))).cuda()
    t = torch.from_numpy(np.stack([np.sin(3 * E + j) for j in range(16)], 1).astype(np.float32)).cuda()
    l0 = net.train_step(x, t, 0.0)
    for _ in range(200):
        net.train_step(x, t, 3e-3)
    l1 = net.train_step(x, t, 0.0)
    assert l1 < 0.2 * l0


def test_warm_start_workload_report(ss, capsys):
    """Lead s_b = 128, 4096 training (E, k) points, 1024 evaluation energies at k = 0."""
    import torch
    from paper_1812_01396_gb300 import warm
    s, nk = 128, 16
    kgrid = np.linspace(0.0, np.pi, nk, endpoint=False)
    devs = synth.make_device(2, s, seed=5, k_points=kgrid, w_scale=0.25)
    h = ss.Handle(n_b_max=2, s_b_max=s, max_points=64, max_inj=1)
    try:
        for i, d in enumerate(devs):
            h.set_device(i, d)
        rng = np.random.default_rng(7)
        n_train = 4096
        Etr = rng.uniform(-1, 1, n_train)
        ktr_id = rng.integers(0, nk, n_train)
        t0 = time.time()
        g_probe, _, _, _, _ = h.surface_gf(Etr[:64], ktr_id[:64], side=1)
        scale = 1.0 / float(np.sqrt(np.mean([np.mean(np.abs(g) ** 2) for g in g_probe])))
        net = ss.MLP(warm.N_IN, 512, 2 * s * s, 256, seed=11)
        losses, _ = warm.train(net, h, Etr, ktr_id, kgrid[ktr_id], 1, scale, epochs=40, batch=256, lr=1e-3)
        t_train = time.time() - t0
        h.set_warm_start(net, 1, scale)
        Ev = -1.0 + (2 * np.arange(1024) + 1) / 1024.0
        kid = np.zeros(1024, np.int32)
        t_plain = t_warm = float("inf")
        for _ in range(2):  # best of two timed calls each
            torch.cuda.synchronize()
            t0 = time.time()
            g0, it0, _, st0, _ = h.surface_gf(Ev, kid, side=1)
            t_plain = min(t_plain, time.time() - t0)
            t0 = time.time()
            g1, it1, seeded, st1, _ = h.surface_gf(Ev, kid, np.zeros(1024), side=1, use_warm=True, warm_iters=8,
                                                   warm_tol=1e-10)
            t_warm = min(t_warm, time.time() - t0)
    finally:
        h.close()
    errs = np.array([rel(a, b) for a, b in zip(g1, g0)])
    acc = seeded.astype(bool)
    # accepted seeds satisfy the Dyson residual test; rejected ones are the doubling itself
    assert np.all(errs[~acc] == 0.0)
    if acc.any():
        assert np.max(errs[acc]) < 1e-6
    report = dict(train_points=n_train, train_seconds=round(t_train, 2), final_loss=losses[-1], first_loss=losses[0],
                  eval_points=1024, accepted=int(acc.sum()), mean_iters_plain=float(it0.mean()),
                  mean_iters_warm=float(np.where(acc, it1, it0 + 8).mean()), t_plain_s=round(t_plain, 3),
                  t_warm_s=round(t_warm, 3), gain_time=round(t_plain / t_warm, 3))
    with capsys.disabled():
        print("\nwarm-start report (in band):", report)
    assert losses[-1] < losses[0]


def test_warm_start_gap_energies_report(ss, capsys):
    """The same lead (s_b = 128) at energies in the gap above its band, where
    every mode decays and the fixed point contracts by |lambda|^2 < 1: a
    network trained there (1024 points) seeds 512 evaluation energies.  Reports
    accepted seeds and time against the plain doubling; checks that every
    accepted g equals the doubling's within the residual bar."""
    import torch
    from paper_1812_01396_gb300 import warm
    s = 128
    dev = synth.make_device(2, s, seed=5)[0]
    h = ss.Handle(n_b_max=2, s_b_max=s, max_points=64, max_inj=1)
    try:
        h.set_device(0, dev)
        rng = np.random.default_rng(9)
        Etr = rng.uniform(40.0, 60.0, 1024)
        g_probe, _, _, _, _ = h.surface_gf(Etr[:64], np.zeros(64, np.int32), side=1)
        scale = 1.0 / float(np.sqrt(np.mean([np.mean(np.abs(g) ** 2) for g in g_probe])))
        net = ss.MLP(warm.N_IN, 512, 2 * s * s, 256, seed=12)
        losses, _ = warm.train(net, h, Etr, np.zeros(1024, np.int32), np.zeros(1024), 1, scale, epochs=30,
                               batch=256, lr=1e-3)
        h.set_warm_start(net, 1, scale)
        Ev = np.linspace(41.0, 59.0, 512)
        kid = np.zeros(512, np.int32)
        # best of three timed calls each (host clock around the synchronous calls)
        t_plain = t_warm = float("inf")
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.time()
            g0, it0, _, st0, _ = h.surface_gf(Ev, kid, side=1)
            t_plain = min(t_plain, time.time() - t0)
            t0 = time.time()
            g1, it1, seeded, st1, _ = h.surface_gf(Ev, kid, np.zeros(512), side=1, use_warm=True, warm_iters=8,
                                                   warm_tol=1e-10)
            t_warm = min(t_warm, time.time() - t0)
    finally:
        h.close()
    errs = np.array([rel(a, b) for a, b in zip(g1, g0)])
    acc = seeded.astype(bool)
    assert np.all(np.asarray(st0) == 0) and np.all(np.asarray(st1) == 0)
    assert np.all(errs[~acc] == 0.0)
    if acc.any():
        assert np.max(errs[acc]) < 1e-9, np.max(errs[acc])
    report = dict(train_points=1024, final_loss=losses[-1], first_loss=losses[0], eval_points=512,
                  accepted=int(acc.sum()), mean_iters_plain=float(it0.mean()), t_plain_s=round(t_plain, 3),
                  t_warm_s=round(t_warm, 3), gain_time=round(t_plain / t_warm, 3))
    with capsys.disabled():
        print("\nwarm-start report (gap):", report)


def test_pipeline_warm_start_accepted_branch(ss):
    """cfg.warm_start inside ss_self_energy / ss_solve: at energies far above the
    band the fixed point contracts by about |lambda|^2 ~ 0.02 per step, so even
    an untrained network's seed (scaled down) passes the 1e-10 Dyson test
    after 8 steps; those leads skip the doubling (iters = -8) and their
    self-energies, T and x must still equal the oracle's.  The in-band point
    is rejected and equals the run without warm start bit for bit."""
    import torch
    dev = synth.make_device(4, 32, seed=21)[0]
    net = ss.MLP(19, 64, 2 * 32 * 32, 8, seed=5)
    Es = [60.0, 0.3, 75.0]
    inj = [synth.make_injection(32, 2, seed=30 + i)[0] for i in range(3)]
    out = {}
    for ws in (0, 1):
        h = ss.Handle(n_b_max=4, s_b_max=32, max_points=3, max_inj=2, warm_start=ws)
        try:
            h.set_device(0, dev)
            h.set_momentum(0, 0.0)
            h.set_warm_start(net, 0, 1e3)
            h.set_warm_start(net, 1, 1e3)
            sL, sR, it, st, _ = h.self_energy(Es, [0, 0, 0])
            xs, stx, _ = h.solve(Es, [0, 0, 0], inj)
            T, err, stT, _ = h.transmission(Es, [0, 0, 0])
        finally:
            h.close()
        out[ws] = dict(sL=sL, sR=sR, it=np.asarray(it), x=xs, T=np.asarray(T), st=np.asarray(stT))
    w, p0 = out[1], out[0]
    assert np.all(w["st"] == 0)
    assert list(w["it"][0]) == [-8, -8] and list(w["it"][2]) == [-8, -8], w["it"]
    assert np.all(w["it"][1] > 0)
    assert np.array_equal(w["sL"][1], p0["sL"][1]) and float(w["T"][1]) == float(p0["T"][1])
    for p in (0, 2):
        ref = dense.solve_point(dev, Es[p], inj[p])
        assert rel(w["sL"][p], ref["sigma_L"]) < 1e-9 and rel(w["sR"][p], ref["sigma_R"]) < 1e-9
        assert rel(w["x"][p], ref["x"]) < 1e-9
        assert dense.rel_T_err(float(w["T"][p]), ref["T"]) < 1e-10

"""Throughput of the SplitSolve hot path on GB300: (E,k) solves/s and TFLOP/s.

Workload (default): nanowire-like FP64 SplitSolve, n_b = 64 blocks of
s_b = 512, sparse-banded blocks (|a-b| <= 25, ~10 % fill), S = I + 0.02
perturbation, 64 energies in [-1, 1] x 4 k-points = 256 (E,k) points, seed 2,
n_inj = 32 injected columns per point.  One step solves one batch of
``--batch`` points of that grid (self-energies, both block sweeps, boundary
correction, x and T) through the C ABI.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (bounded sample: one (E,k) point per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "(E,k) solves/s and TFLOP/s vs peak; mixed vs FP64 at rel T err<=1e-8"
FP64_NOMINAL_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--n_b", type=int, default=64)
    ap.add_argument("--s_b", type=int, default=512)
    ap.add_argument("--n_inj", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(a):
    devs = synth.make_device(a.n_b, a.s_b, seed=2, band=25, s_pert=0.02, k_points=synth.K_POINTS_4,
                             w_scale=0.25)
    E = synth.energy_grid(64)
    pts = [(float(e), k) for k in range(4) for e in E]   # 256 points, (E, k_id)
    return devs, pts


def wl_name(a):
    return (f"nanowire-like FP64 SplitSolve: n_b={a.n_b}, s_b={a.s_b}, banded ~10% fill, "
            f"64 E x 4 k = 256 (E,k) points, {a.batch} points per step, n_inj={a.n_inj}")


def point_flops(n, s, ninj, itL, itR):
    """Algorithmic flops of one point (complex MAC = 8, zgetrf = 8/3 s^3)."""
    s3 = float(s) ** 3
    dec = (itL + itR) * (8 / 3 + 16 + 32) * s3 + 2 * (8 / 3 + 8 + 8) * s3
    sweeps = 2 * (n * (8 / 3 + 8) * s3 + (n - 1) * 16 * s3)
    s2i = float(s) ** 2 * ninj
    bound = 32 * s3 + 48 * s2i + 8 / 3 * 8 * s3 + 32 * s3 + 32 * s2i + 16 * s3 + 16 * n * s2i + 16 * s3
    return dec + sweeps + bound


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_point(dev, E, inj):
    from oracle import rgf
    return rgf.solve_point(dev, E, inj)


def cpu_baseline(devs, pts, inj, budget_s=30.0):
    """Oracle (RGF + doubling, FP64 numpy on the host cores) on a bounded sample."""
    t0 = time.perf_counter()
    done = 0
    for (E, k) in pts:
        oracle_point(devs[k], E, inj)
        done += 1
        if time.perf_counter() - t0 > budget_s * 0.5:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "(E,k) solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} (E,k) point(s) of the workload, FP64 numpy RGF + Sancho-Rubio doubling, "
                      f"{dt:.1f} s"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    devs, pts = workload(a)
    inj = synth.make_injection(a.s_b, a.n_inj, seed=2)[0]
    for i in range(a.warmup):
        E, k = pts[i % len(pts)]
        oracle_point(devs[k], E, inj)
    t0 = time.perf_counter()
    for i in range(a.steps):
        E, k = pts[(a.warmup + i) % len(pts)]
        oracle_point(devs[k], E, inj)
    dt = time.perf_counter() - t0
    v = a.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "(E,k) solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_name(a) + " (oracle: one point per step)"},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": v,
                             "sample": "one (E,k) point per step, FP64 numpy RGF + doubling"},
            "e2e": {"value": v, "unit": "(E,k) solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_gemm_peak(torch):
    """cuBLAS DGEMM 8192^3 throughput (TFLOP/s), best of 5."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = max(best, 2 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b
    torch.cuda.empty_cache()
    return best


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import torch
    import torch.distributed as dist

    import paper_1812_01396_gb300 as ss

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    devs, pts = workload(a)
    stream = torch.cuda.Stream()
    P = a.batch
    h = ss.Handle(n_b_max=a.n_b, s_b_max=a.s_b, max_points=P, max_inj=a.n_inj, device_ptrs=1,
                  stream=stream.cuda_stream)
    tdev = []
    with torch.cuda.stream(stream):
        for k, d in enumerate(devs):
            t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", non_blocking=False)
            h.set_hamiltonian(k, t(d.H_diag), t(d.H_up), t(d.S_diag), t(d.S_up))
        inj_host = synth.make_injection(a.s_b, a.n_inj, seed=2, n_pts=P)
        inj_dev = torch.from_numpy(inj_host).cuda()
    stream.synchronize()

    # this rank's points: a strided slice of the grid, P per step
    mine = pts[rank::world]

    def batch(step):
        sel = [mine[(step * P + i) % len(mine)] for i in range(P)]
        return [e for e, _ in sel], [k for _, k in sel]

    def step(hh, s, inj, want_x=True):
        E, K = batch(s)
        _, _, it, st0, _ = hh.self_energy(E, K)
        xs, st1, _ = hh.solve(E, K, inj, want_x=want_x)
        T, err, st2, _ = hh.transmission(E, K)
        return it, T, np.maximum(np.maximum(st0, st1), st2)

    with torch.cuda.stream(stream):
        for s in range(a.warmup):
            step(h, s, inj_dev)
    stream.synchronize()

    # ---- timed region (device-resident inputs)
    launches0 = h.launch_count()
    flops = 0.0
    iters = []
    clk = Clocks(os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else ".",
                              f"clocks_rank{rank}.csv"))
    barrier()
    torch.cuda.synchronize()
    with clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for s in range(a.warmup, a.warmup + a.steps):
                it, T, st = step(h, s, inj_dev)
                iters.append(it)
        e1.record(stream)
        e1.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_dev = e0.elapsed_time(e1) * 1e-3
    launches = h.launch_count() - launches0
    for it in iters:
        for p in range(P):
            flops += point_flops(a.n_b, a.s_b, a.n_inj, int(it[p, 0]), int(it[p, 1]))
    t_max = t_dev
    if world > 1:
        tt = torch.tensor([t_dev], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    n_solved = P * a.steps * world
    value = n_solved / t_max

    # ---- profiled pass (same steps): per-kernel device time with CUDA events
    hp = ss.Handle(n_b_max=a.n_b, s_b_max=a.s_b, max_points=P, max_inj=a.n_inj, device_ptrs=1,
                   stream=stream.cuda_stream, profile=1)
    with torch.cuda.stream(stream):
        for k, d in enumerate(devs):
            t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
            hp.set_hamiltonian(k, t(d.H_diag), t(d.H_up), t(d.S_diag), t(d.S_up))
        step(hp, 0, inj_dev)
        hp.profile_reset()
        for s in range(a.warmup, a.warmup + a.steps):
            step(hp, s, inj_dev)
    stream.synchronize()
    kern = {}
    for name in ss.KERNEL_KINDS:
        ms, fl, n = hp.profile_read(name)
        kern[name] = {"ms": ms, "launches": n, "flops": fl}
    hp.close()
    tot_ms = sum(v["ms"] for v in kern.values()) or 1.0
    g = kern["zgemm"]
    peak_meas = fp64_gemm_peak(torch)
    achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_meas, "unit": "TFLOP/s",
                "frac": achieved / peak_meas if peak_meas else None, "traffic": None,
                "kernel": "zgemm_kernel (FP64 DFMA complex GEMM)",
                "peak_source": "measured cuBLAS DGEMM 8192^3 on this GPU (FP64 pipe); nominal 1.25",
                "avg_launch_ms": g["ms"] / max(g["launches"], 1),
                "share_of_kernel_time": g["ms"] / tot_ms}

    # ---- end to end through host buffers (pinned), copies inside the timed region
    e2e = None
    if not a.no_e2e:
        he = ss.Handle(n_b_max=a.n_b, s_b_max=a.s_b, max_points=P, max_inj=a.n_inj, device_ptrs=0,
                       stream=stream.cuda_stream)
        for k, d in enumerate(devs):
            he.set_device(k, d)
        pinned = torch.from_numpy(inj_host).pin_memory().numpy()
        inj_list = [pinned[i] for i in range(P)]
        with torch.cuda.stream(stream):
            step(he, 0, inj_list)
        stream.synchronize()
        barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for s in range(a.warmup, a.warmup + a.steps):
                step(he, s, inj_list)
        stream.synchronize()
        te = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([te], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        he.close()
        h2d = P * 2 * a.s_b * a.n_inj * 16
        d2h = P * a.n_b * a.s_b * a.n_inj * 16 + P * 8
        e2e = {"value": n_solved / te, "unit": "(E,k) solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank == 0:
        cpu = None
        if not a.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(devs, pts, inj_host[0])
        line = {
            "metric": METRIC, "value": value, "unit": "(E,k) solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * t_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_name(a), "n_b": a.n_b, "s_b": a.s_b, "points_per_step": P,
                       "n_inj": a.n_inj, "precision": "fp64", "parallelism": f"(E,k) shards x{world}",
                       "l2": "inputs larger than L2: per-step workspace "
                             f"{P * (2 * a.n_b + 43) * a.s_b ** 2 * 16 / 1e9:.1f} GB"},
            "tflops": flops * world / t_max / 1e12,
            "roofline": roofline,
            "kernels_ms": {k: round(v["ms"], 3) for k, v in kern.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "status_ok": bool(np.all(st == 0)),
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

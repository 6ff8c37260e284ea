"""Sharding of (E,k) points over ranks, one process per GPU.

Every (E,k) point is an independent solve (the points of a spectrum are
"almost embarrassingly parallel", Sec. 4), so a multi-GPU run only partitions
the points and gathers one transmission per point at the end; no collective
sits on the data path.  Uneven batches are balanced by longest-processing-time
first over the per-point cost model of the hot path.
"""
from __future__ import annotations

import numpy as np

# Per-point cost in units of s_b^3 complex-FP64 flops / 8: sweeps of both
# block columns (Algorithm 1 and its mirror, about 53.3 n_b s_b^3 real flops)
# plus the doubling of both leads (about 2 * iters * 59 s_b^3).
SWEEP_PER_BLOCK = 53.3
DOUBLING_PER_STEP = 2 * 59.0


def point_cost(n_b: int, s_b: int, doubling_steps: int = 40) -> float:
    """Relative work of one (E,k) point of a device with n_b blocks of size s_b."""
    return (SWEEP_PER_BLOCK * n_b + DOUBLING_PER_STEP * doubling_steps) * float(s_b) ** 3


def strided_shard(n_points: int, rank: int, world: int) -> list[int]:
    """Points rank, rank + world, ... (equal-cost points)."""
    return list(range(rank, n_points, world))


def lpt_shard(costs, world: int) -> list[list[int]]:
    """Longest processing time first: points by decreasing cost, each to the
    least-loaded rank (lowest rank on ties).  Returns the point indices of
    every rank, each list in increasing order.  Deterministic, so every rank
    computes the same partition without communicating."""
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = np.zeros(world)
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(load))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_values(values, indices, n_points: int) -> np.ndarray:
    """Every rank's (index, value) pairs gathered into one array of n_points
    (host gather over the default process group; NaN where no rank wrote)."""
    import torch
    import torch.distributed as dist

    dev = _comm_device()
    local = torch.tensor(np.stack([np.asarray(indices, np.float64), np.asarray(values, np.float64)], 1)
                         if len(indices) else np.zeros((0, 2)), dtype=torch.float64, device=dev)
    world = dist.get_world_size()
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([local.shape[0]], dtype=torch.int64, device=dev))
    cap = int(max(int(s) for s in sizes))
    pad = torch.full((cap, 2), float("nan"), dtype=torch.float64, device=dev)
    pad[:local.shape[0]] = local
    bufs = [torch.empty((cap, 2), dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(bufs, pad)
    out = np.full(n_points, np.nan)
    for b, n in zip(bufs, sizes):
        b = b[:int(n)].cpu().numpy()
        out[b[:, 0].astype(np.int64)] = b[:, 1]
    return out


def _comm_device():
    """Tensors of a host-side exchange live on the GPU under NCCL, on the host under gloo."""
    import torch
    import torch.distributed as dist

    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(v: float) -> float:
    """The largest value over all ranks (step times: the job takes the slowest)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=_comm_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

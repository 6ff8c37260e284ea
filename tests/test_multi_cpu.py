"""Multi-process host logic of the N-GPU path, on CPU ranks (gloo, world 2):
the LPT partition covers every point once and is balanced, the gather
rebuilds the serial result (the oracle's T of every point of an uneven batch,
each computed on the rank LPT gave it), and the step time is the maximum over
ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1812_01396_gb300 import multi

import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _points():
    pts = synth.uneven_points(37, seed=3)
    return pts, [multi.point_cost(n, s) for (s, n, _, _) in pts]


def _small_points():
    """Uneven small points (s_b, n_b, E, k) whose oracle T a CPU rank computes in
    milliseconds: the same kind of work a GPU rank shards, at a tenth of the size."""
    pts = synth.uneven_points(14, seed=5, s_choices=(4, 6, 8), n_choices=(2, 3, 5))
    return pts, [multi.point_cost(n, s) for (s, n, _, _) in pts]


def _oracle_T(pt):
    from oracle import dense
    s, n, E, k = pt
    dev = synth.make_device(n, s, seed=100 + 7 * s + n, k_points=(k,), w_scale=0.25)[0]
    return float(dense.solve_point(dev, E)["T"])


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts, costs = _small_points()
        mine = multi.lpt_shard(costs, world)[rank]
        T = [_oracle_T(pts[i]) for i in mine]
        full = multi.gather_values(T, mine, len(pts))
        slowest = multi.max_over_ranks(1.0 + rank)
        if rank == 0:
            out.put((full.tolist(), slowest))
    finally:
        dist.destroy_process_group()


def test_lpt_partition_covers_once_and_balances():
    pts, costs = _points()
    for world in (1, 2, 3, 8):
        parts = multi.lpt_shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(pts)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT guarantee: the spread is at most the largest single cost
        assert max(loads) - min(loads) <= max(costs) + 1e-9
    assert multi.strided_shard(10, 1, 3) == [1, 4, 7]


def test_gather_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    full, slowest = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pts, _ = _small_points()
    ref = [_oracle_T(pt) for pt in pts]
    assert np.array_equal(np.asarray(full), np.asarray(ref))  # same arithmetic on every rank: bit-equal
    assert slowest == 2.0

"""Sharded ensemble statistics on two CPU ranks (gloo): the per-rank partial projections and
Monte Carlo moments merged across ranks equal the unsharded oracle statistics."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import uq as ouq
from paper_2508_13867_gb300 import shard
from paper_2508_13867_gb300 import workloads as W


def test_partition_balances_work_and_covers_all_samples():
    specs = W.uneven_batch(n_tgv=40, n_cyl=8)
    costs = shard.sample_costs(specs)
    for world in (1, 2, 3, 8):
        blocks = shard.partition(costs, world)
        assert blocks[0][0] == 0 and blocks[-1][1] == len(costs)
        assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
        loads = [sum(costs[a:b]) for a, b in blocks]
        assert max(loads) - min(loads) <= max(costs) + 1e-9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bounds = W.TGV4D_BOUNDS
        _, xi, a = ouq.tensor_grid([3] * 4, bounds)
        alpha = ouq.multi_indices(4, 2)
        m = W.random_fields(len(a), 257, seed=9)
        lo, hi = shard.partition(np.ones(len(a)), world)[rank]
        wmat = ouq.weight_matrix(alpha, xi, a)
        part = torch.from_numpy(wmat[:, lo:hi] @ m[lo:hi])
        coeffs = shard.merge_gpc_coefficients(part).numpy()
        blk = m[lo:hi]
        mean = torch.from_numpy(blk.mean(axis=0))
        m2 = torch.from_numpy(((blk - blk.mean(axis=0)) ** 2).sum(axis=0))
        n, mu, q2 = shard.merge_mc_moments(hi - lo, mean, m2)
        q.put((rank, coeffs, n, mu.numpy(), q2.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_matches_unsharded_oracle():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    bounds = W.TGV4D_BOUNDS
    _, xi, a = ouq.tensor_grid([3] * 4, bounds)
    m = W.random_fields(len(a), 257, seed=9)
    c_ref = ouq.gpc_coefficients(ouq.multi_indices(4, 2), xi, a, m)
    mean_ref, var_ref = ouq.mc_mean_var(m, ddof=1)
    for rank, coeffs, n, mu, q2 in out:
        assert np.allclose(coeffs, c_ref, rtol=1e-13, atol=1e-15), rank
        assert n == len(a)
        assert np.allclose(mu, mean_ref, rtol=1e-14, atol=0)
        assert np.allclose(q2 / (n - 1), var_ref, rtol=1e-12, atol=0)

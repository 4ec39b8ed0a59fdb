"""Sharded ensemble statistics on two CPU ranks (gloo): the per-rank partial projections and
Monte Carlo moments merged across ranks equal the unsharded oracle statistics.  Each rank takes its
block from the library's partition helper and the block's weight columns from the library
(uqlb_get_weight_block, the matrix that uqlb_project_block uploads); the product with the block's
fields, which the library forms on the GPU, is formed here on the host (the GPU half is covered by
the sample-block test of the GPU suite)."""
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
    from paper_2508_13867_gb300 import uqlb as U

    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_gpc(ctx, 2, 3)
        S = U.uqlb_num_samples(ctx)
        m = W.random_fields(S, 257, seed=9)
        lo, hi = shard.partition(np.ones(S), world)[rank]
        wblk = U.uqlb_get_weight_block(ctx, lo, hi - lo)
        part = torch.from_numpy(wblk @ m[lo:hi])
        coeffs = shard.merge_gpc_coefficients(part).numpy()
        blk = m[lo:hi]
        mean = torch.from_numpy(blk.mean(axis=0))
        m2 = torch.from_numpy(((blk - blk.mean(axis=0)) ** 2).sum(axis=0))
        n, mu, q2 = shard.merge_mc_moments(hi - lo, mean, m2)
        q.put((rank, coeffs, n, mu.numpy(), q2.numpy()))
    finally:
        U.uqlb_destroy(ctx)
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


def test_weight_blocks_tile_the_weight_matrix():
    """The columns a block projection uploads are the block's columns of W, and blocks that cover
    the samples reassemble W; blocks outside the sample set are refused."""
    from paper_2508_13867_gb300 import uqlb as U

    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_gpc(ctx, 4, 3)
        S = U.uqlb_num_samples(ctx)
        full = U.uqlb_get_weight_matrix(ctx)
        for world in (1, 2, 5):
            parts = [U.uqlb_get_weight_block(ctx, lo, hi - lo) for lo, hi in shard.partition(np.ones(S), world)]
            assert np.array_equal(np.concatenate(parts, axis=1), full)
        for lo, n in ((-1, 2), (S - 1, 2), (0, 0)):
            with pytest.raises(U.UqlbError) as e:
                U.uqlb_get_weight_block(ctx, lo, n)
            assert e.value.status == U.UQLB_ERR_ARG
    finally:
        U.uqlb_destroy(ctx)


def test_chan_merge_of_blocks_equals_the_whole():
    """The in-order pairwise merge of block moments equals the moments of the whole set (uneven
    blocks, an empty block)."""
    m = W.random_fields(101, 33, seed=4)
    cuts = [0, 7, 7, 50, 101]
    blocks = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        blk = torch.from_numpy(m[a:b])
        mean = blk.mean(0) if b > a else torch.zeros(33, dtype=torch.float64)
        blocks.append((b - a, mean, ((blk - mean) ** 2).sum(0)))
    n, mu, q2 = shard.chan_merge(blocks)
    mr, vr = ouq.mc_mean_var(m, ddof=1)
    assert n == 101
    assert np.allclose(mu.numpy(), mr, rtol=1e-14, atol=0)
    assert np.allclose(q2.numpy() / 100, vr, rtol=1e-12, atol=0)

"""Sample sharding across ranks (one process per GPU) and the merge of per-rank statistics.

The ensemble's samples are independent (Sec. 7, sample-level parallelism), so a sharded run
gives every rank a contiguous block of samples balanced by lattice work (nodes x steps).  The
only exchange is at the end:
  * gPC: coefficients are linear in the samples, c_k = sum_s W[k, s] M[s, :], so each rank
    projects its own columns of W and the partial coefficients are summed (one all-reduce);
  * MC: each rank reduces (n, mean, M2) of its block and the blocks are combined with the
    pairwise update of Chan, Golub and LeVeque, in rank order so the result does not depend on
    arrival order.
The merge functions run on torch tensors of any device; with world size 1 they are identities.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def partition(costs, world: int) -> list[tuple[int, int]]:
    """Contiguous blocks [lo, hi) of samples, one per rank, with near-equal summed cost."""
    costs = np.asarray(costs, dtype=np.float64)
    n = len(costs)
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target, side="left"))
        k = min(max(k, cuts[-1]), n)
        # pick the nearer of the two cut points around the target
        if 0 < k <= n and abs(cum[k - 1] - target) < abs(cum[k] - target) and k - 1 >= cuts[-1]:
            k -= 1
        cuts.append(k)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def sample_costs(samples) -> list[int]:
    """Lattice work of each sample: nodes x steps."""
    return [int(s.nx) * int(s.ny) * int(s.steps) for s in samples]


def _world() -> int:
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def merge_gpc_coefficients(partial: torch.Tensor) -> torch.Tensor:
    """Sum the per-rank partial coefficients (in place) and return them."""
    if _world() > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM)
    return partial


def chan_merge(blocks):
    """Combine (count, mean, sum of squared deviations) of consecutive sample blocks, in order, by
    the pairwise update of Chan, Golub and LeVeque.  Returns (N, mean, M2)."""
    na, ma, qa = blocks[0][0], blocks[0][1].clone(), blocks[0][2].clone()
    for nb, mb, qb in blocks[1:]:
        if nb == 0:
            continue
        nt = na + nb
        delta = mb - ma
        ma = ma + delta * (nb / nt)
        qa = qa + qb + delta * delta * (na * nb / nt)
        na = nt
    return int(na), ma, qa


def merge_mc_moments(n: int, mean: torch.Tensor, m2: torch.Tensor):
    """Combine per-rank (count, mean, sum of squared deviations) into the global ones, in rank order.

    Returns (N, mean, M2); the variance with divisor N - ddof is M2 / (N - ddof)."""
    world = _world()
    if world == 1:
        return n, mean, m2
    counts = [torch.zeros(1, dtype=torch.float64, device=mean.device) for _ in range(world)]
    means = [torch.empty_like(mean) for _ in range(world)]
    m2s = [torch.empty_like(m2) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([float(n)], dtype=torch.float64, device=mean.device))
    dist.all_gather(means, mean.contiguous())
    dist.all_gather(m2s, m2.contiguous())
    return chan_merge([(float(counts[r].item()), means[r], m2s[r]) for r in range(world)])


def run_block(ens, w, rank: int, world: int, storage: str | None = None, fields_dtype: str = "f32", ddof: int = 1,
              out: dict | None = None) -> dict:
    """The sharded UQ pass of one rank: its block of the workload's samples through the library
    (run, then the block projection or block moments), the one exchange, and the statistics.
    `ens` has been set up for the workload (the full sample set); returns the block's outputs and
    the merged mean and variance fields (on every rank)."""
    smp = ens.ensemble_samples(w)
    lo, hi = partition(sample_costs(smp), world)[rank]
    res = ens.run_batch(smp[lo:hi], storage=storage or w.storage, fields_dtype=fields_dtype, qoi_every=w.qoi_every,
                        out=out)
    m = res["fields"]
    if w.method == "gpc":
        coeffs = merge_gpc_coefficients(ens.project_block(m, lo, res.get("coeffs")))
        res["coeffs"] = coeffs
        res["mean"], res["var"] = ens.stats(coeffs)
    else:
        n, mean, m2 = merge_mc_moments(*ens.block_moments(m))
        res["mean"], res["var"] = mean, m2 / (n - ddof)
    res["block"] = (lo, hi)
    return res

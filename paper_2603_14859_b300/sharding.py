"""Voxel sharding across ranks (one process per GPU).

The path partitions by voxels: every rank regenerates the same seeded prior
draws (same Philox seed, same input function) and works on its own voxel
shard, so no collective touches the data path.  The only collective is the
max-over-ranks of the timings that the benchmark reports.
"""
from __future__ import annotations

from . import synth as S


def rank_workload(name: str, rank: int, J: int | None = None, N_per_model: int | None = None) -> S.Workload:
    """Rank `rank`'s voxel shard of workload `name`: rank 0 holds the named volume,
    rank r > 0 an independent volume of the same shape (voxel seed 5000 + r) that
    shares rank 0's draws (prior seed) and input function."""
    W = S.workload(name, seed=None, J=J, N_per_model=N_per_model)
    if rank == 0:
        return W
    Wr = S.workload(name, seed=5000 + rank, J=J, N_per_model=N_per_model)
    Wr.prior_seed = W.prior_seed
    Wr.inp = W.inp
    Wr.model_inp = W.model_inp
    return Wr


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]

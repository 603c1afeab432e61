"""Voxel sharding across ranks (one process per GPU).

The path partitions by voxels: every voxel's accepted set depends only on its own
TAC and the draws, so ranks that regenerate the same seeded prior draws (same
Philox seed, same input function) and each take a disjoint voxel range of the
volume need no collective on the data path.  The only collective is the
max-over-ranks of the timings that the benchmark reports.

A volume is a sequence of blocks of one workload's shape: block 0 is the named
workload itself, block b > 0 the same workload generated with voxel seed
(seed + 7919 b) but sharing block 0's draws and input functions, so that any voxel
range can be generated without the rest.  Weak scaling: rank r takes block r of a
volume of `world` blocks.  Strong scaling: the ranks split block 0 into contiguous
voxel ranges.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import synth as S

BLOCK_SEED_STRIDE = 7919


def voxel_range(J: int, rank: int, world: int) -> tuple[int, int]:
    """Rank `rank`'s share [j0, j1) of J voxels split into `world` contiguous ranges."""
    base, extra = divmod(J, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def volume_block(name: str, b: int, J: int | None = None, N_per_model: int | None = None) -> S.Workload:
    """Block b of the volume of workload `name` (block 0 is the workload itself)."""
    W0 = S.workload(name, seed=None, J=J, N_per_model=N_per_model)
    if b == 0:
        return W0
    base_seed = W0.prior_seed - 7           # the workload's voxel seed (prior seed = seed + 7)
    Wb = S.workload(name, seed=base_seed + BLOCK_SEED_STRIDE * b, J=J, N_per_model=N_per_model)
    Wb.prior_seed = W0.prior_seed
    Wb.inp = W0.inp
    Wb.model_inp = W0.model_inp
    return Wb


def voxel_subset(W: S.Workload, j0: int, j1: int) -> S.Workload:
    """The workload restricted to voxels [j0, j1) (same draws, inputs and noise model).
    Gaussian noise only: Poisson counting noise is drawn for a whole volume at once."""
    if W.noise != "gaussian":
        raise NotImplementedError("voxel ranges of a Poisson-noise workload")
    truth, rows = [], []
    for th, r in zip(W.truth, W.truth_rows):
        r = np.asarray(r)
        keep = (r >= j0) & (r < j1)
        truth.append(th[keep])
        rows.append(r[keep] - j0)
    return dataclasses.replace(W, truth_model=W.truth_model[j0:j1], truth=truth, truth_rows=rows, q=W.q[j0:j1],
                               z=W.z[j0:j1])


def rank_workload(name: str, rank: int, world: int = 1, J: int | None = None, N_per_model: int | None = None,
                  scaling: str = "weak") -> S.Workload:
    """Rank `rank`'s voxel shard: block `rank` of the volume (weak scaling: every rank holds
    a full-size block), or its contiguous range of block 0 (strong scaling)."""
    if scaling == "weak":
        return volume_block(name, rank, J=J, N_per_model=N_per_model)
    if scaling != "strong":
        raise ValueError(scaling)
    W = volume_block(name, 0, J=J, N_per_model=N_per_model)
    return voxel_subset(W, *voxel_range(W.J, rank, world))


def sum_over_ranks(value, dist=None, device=None):
    """Sum of one number over all ranks (identity without a process group)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.cpu()[0])


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]

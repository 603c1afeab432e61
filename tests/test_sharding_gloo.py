"""The multi-rank path on CPU: two gloo ranks shard the voxels, regenerate the
same draws, compute their shards independently (the FP64 oracle stands in for
the device path here) and agree on the max-over-ranks timing; the union of the
shard results equals what one process computes for both shards."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2603_14859_b300 import sharding
    from paper_2603_14859_b300 import synth as S
    W = sharding.rank_workload("brain_fdg_2tcm", rank, J=24, N_per_model=400)
    # the draws every rank regenerates
    lo, hi = W.priors(S.TCM2_IRR)
    th = oracle.sample_prior(W.prior_seed, S.TCM2_IRR, lo, hi, W.N)
    x = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, th)
    # this rank's voxels
    xc = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, W.truth[0])
    y = S.add_noise(xc, W.ts, W.te, W.half_life, W.q, W.z)
    idx, dist_ = oracle.topk(y, x, W.weights, 10)
    t = sharding.max_over_ranks([1.0 + rank, 5.0 - rank], dist)
    obj = [None] * world
    dist.all_gather_object(obj, dict(rank=rank, seed=W.prior_seed, theta0=th[:3].tolist(), y0=y[0].tolist(),
                                     idx=idx.tolist(), t=t))
    if rank == 0:
        out.put(obj)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_voxels_and_share_draws():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = out.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = res
    assert a["seed"] == b["seed"] and a["theta0"] == b["theta0"]         # same draws on every rank
    assert a["y0"] != b["y0"]                                           # different voxel shards
    assert a["t"] == b["t"] == [2.0, 5.0]                               # max over ranks
    # the shards' results are what one process computes for each shard
    import oracle
    from paper_2603_14859_b300 import sharding
    from paper_2603_14859_b300 import synth as S
    for r, got in enumerate(res):
        W = sharding.rank_workload("brain_fdg_2tcm", r, J=24, N_per_model=400)
        lo, hi = W.priors(S.TCM2_IRR)
        x = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, oracle.sample_prior(W.prior_seed, S.TCM2_IRR, lo, hi, W.N))
        xc = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, W.truth[0])
        y = S.add_noise(xc, W.ts, W.te, W.half_life, W.q, W.z)
        idx, _ = oracle.topk(y, x, W.weights, 10)
        assert np.array_equal(np.array(got["idx"]), idx)


def test_max_over_ranks_without_process_group():
    from paper_2603_14859_b300 import sharding
    assert sharding.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]

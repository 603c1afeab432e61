"""The multi-rank path on CPU (gloo, two ranks, 127.0.0.1).

Each rank takes its shard with the same function the benchmark uses
(sharding.rank_workload): a contiguous voxel range of one volume (strong scaling)
or one block of a volume of blocks (weak scaling).  Every rank regenerates the same
seeded draws and computes its shard on its own (the FP64 oracle stands in for the
device path, which needs a GPU); the ranks agree on the max-over-ranks timing and
on the number of voxels processed; the union of the shards' accepted sets equals
what one process computes for the whole volume."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

J_VOL, N_DRAWS, K = 37, 400, 10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _shard_result(W):
    import oracle
    from paper_2603_14859_b300 import synth as S
    lo, hi = W.priors(S.TCM2_IRR)
    th = oracle.sample_prior(W.prior_seed, S.TCM2_IRR, lo, hi, W.N)
    x = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, th)
    xc = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, W.truth[0])
    y = S.add_noise(xc, W.ts, W.te, W.half_life, W.q, W.z)
    idx, _ = oracle.topk(y, x, W.weights, K)
    return th, idx


def _rank(rank, world, port, scaling, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2603_14859_b300 import sharding
    W = sharding.rank_workload("brain_fdg_2tcm", rank, world, J=J_VOL, N_per_model=N_DRAWS, scaling=scaling)
    th, idx = _shard_result(W)
    t = sharding.max_over_ranks([1.0 + rank, 5.0 - rank], dist)
    n = sharding.sum_over_ranks(W.J, dist)
    obj = [None] * world
    dist.all_gather_object(obj, dict(rank=rank, J=W.J, theta0=th[:3].tolist(), idx=idx.tolist(), t=t, n=n))
    if rank == 0:
        out.put(obj)
    dist.barrier()
    dist.destroy_process_group()


def _run(scaling, world=2):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, scaling, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = out.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def test_strong_scaling_ranks_partition_one_volume():
    from paper_2603_14859_b300 import sharding
    res = _run("strong")
    a, b = res
    assert a["theta0"] == b["theta0"]                                    # same draws on every rank
    assert a["t"] == b["t"] == [2.0, 5.0]                                # max over ranks
    assert a["n"] == b["n"] == J_VOL and a["J"] + b["J"] == J_VOL        # the ranges cover the volume once
    assert sharding.voxel_range(J_VOL, 0, 2) == (0, a["J"]) and sharding.voxel_range(J_VOL, 1, 2) == (a["J"], J_VOL)
    # the union of the shards is what one process computes for the whole volume
    _, whole = _shard_result(sharding.volume_block("brain_fdg_2tcm", 0, J=J_VOL, N_per_model=N_DRAWS))
    assert np.array_equal(np.concatenate([np.array(a["idx"]), np.array(b["idx"])]), whole)


def test_weak_scaling_ranks_take_blocks_of_one_volume():
    from paper_2603_14859_b300 import sharding
    res = _run("weak")
    a, b = res
    assert a["theta0"] == b["theta0"]                                    # blocks share the draws
    assert a["n"] == b["n"] == 2 * J_VOL
    for r, got in enumerate(res):
        _, idx = _shard_result(sharding.volume_block("brain_fdg_2tcm", r, J=J_VOL, N_per_model=N_DRAWS))
        assert np.array_equal(np.array(got["idx"]), idx)
    assert a["idx"] != b["idx"]                                          # different voxels


def test_voxel_ranges_and_subsets():
    from paper_2603_14859_b300 import sharding
    for J in (1, 7, 37, 1000):
        for world in (1, 2, 3, 8):
            rngs = [sharding.voxel_range(J, r, world) for r in range(world)]
            assert rngs[0][0] == 0 and rngs[-1][1] == J
            assert all(rngs[i][1] == rngs[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in rngs) - min(b - a for a, b in rngs) <= 1
    W = sharding.volume_block("raclopride_lpntpet", 0, J=500, N_per_model=10)
    sub = sharding.voxel_subset(W, 120, 340)
    assert sub.J == 220 and np.array_equal(sub.z, W.z[120:340]) and np.array_equal(sub.q, W.q[120:340])
    for (th, rows), (ths, rs) in zip(zip(W.truth, W.truth_rows), zip(sub.truth, sub.truth_rows)):
        keep = (np.asarray(rows) >= 120) & (np.asarray(rows) < 340)
        assert np.array_equal(ths, th[keep]) and np.array_equal(rs + 120, np.asarray(rows)[keep])


def test_max_over_ranks_without_process_group():
    from paper_2603_14859_b300 import sharding
    assert sharding.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert sharding.sum_over_ranks(4) == 4.0

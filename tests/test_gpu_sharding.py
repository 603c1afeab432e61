"""The library on voxel shards of one volume: calls on disjoint voxel ranges (strong
scaling) return, voxel for voxel, what one call on the whole volume returns (each
voxel's accepted set depends only on its TAC and the draws), in every precision form."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_shards_equal_the_whole_volume(prec):
    from paper_2603_14859_b300 import pipeline, sharding
    name, J, n = "raclopride_lpntpet", 3000, 40_000
    W = sharding.volume_block(name, 0, J=J, N_per_model=n)
    whole = pipeline.AbcPipeline(W, prec)
    out = whole.step(pipeline.make_y_gpu(W))
    ref = [t.clone() for t in (out.idx, out.dist, out.prob, out.pref, out.mean, out.sd, out.lo, out.hi)]
    world = 3
    got = []
    for r in range(world):
        Ws = sharding.rank_workload(name, r, world, J=J, N_per_model=n, scaling="strong")
        run = pipeline.AbcPipeline(Ws, prec)
        o = run.step(pipeline.make_y_gpu(Ws))
        got.append([t.clone() for t in (o.idx, o.dist, o.prob, o.pref, o.mean, o.sd, o.lo, o.hi)])
    torch.cuda.synchronize()
    for c in range(len(ref)):
        cat = torch.cat([g[c] for g in got])
        assert torch.equal(torch.nan_to_num(cat, nan=-1.0), torch.nan_to_num(ref[c], nan=-1.0)), f"output {c}"

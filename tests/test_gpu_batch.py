"""Batched uneven scans (many scans in one persistent launch, CUDA graph,
autotuned tiles): every scan must get exactly what its own
abc_discrepancy_topk call returns, which the single-scan tests tie to the
FP64 oracle; one scan of each model family is also checked against the oracle
directly (Alg. 1 steps 4-5)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_14859_b300 import synth as S
from parity import check_topk_sets

pytestmark = pytest.mark.gpu


def _small_plan(n=7):
    plan = S.scan_plan(seed=77, n_scans=n, voxel_scale=0.004, draw_scale=0.01)
    plan[0]["J"] = 1                       # a one-voxel scan
    plan[1]["J"] = 129                     # one full tile plus one voxel
    return plan


@pytest.fixture(scope="module")
def batch(orc):
    from paper_2603_14859_b300 import pipeline
    scans = [S.scan_workload(p, k=40) for p in _small_plan()]
    ys = []
    for W in scans:
        xc = np.zeros((W.J, W.L))
        for model, rows, th in pipeline.truth_groups(W):
            xc[rows] = orc.simulate(model, W.ts, W.te, W.input_for(model), th)
        y = S.add_noise(xc, W.ts, W.te, W.half_life, W.q, W.z)
        ld = (W.L + 3) // 4 * 4
        yp = np.zeros((W.J, ld), np.float32)
        yp[:, :W.L] = y
        ys.append(torch.from_numpy(yp).cuda())
    return scans, ys


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_equals_single_scan_calls(batch, prec):
    from paper_2603_14859_b300 import api, pipeline
    scans, ys = batch
    bp = pipeline.BatchPipeline(scans, prec)
    for r in bp.runs:
        r.simulate_draws()
    bp.set_inputs(ys)
    bp.ws.fill_(0xFF)                                  # stale workspace contents must not matter
    bp.topk()
    torch.cuda.synchronize()
    st = api.topk_status(bp.ws)
    assert st[0] == 0 and st[2] == 0
    for r, y in zip(bp.runs, ys):
        idx, dist = api.discrepancy_topk(y, r.x, r.L, r.weights, r.k, prec)
        assert torch.equal(idx, r.idx), f"{r.W.name}: accepted draws differ from the single-scan call"
        assert torch.equal(dist, r.dist)


@pytest.mark.parametrize("prec", [0, 2])
def test_batch_oracle_parity(batch, orc, prec):
    from paper_2603_14859_b300 import pipeline
    scans, ys = batch
    bp = pipeline.BatchPipeline(scans, prec)
    for r in bp.runs:
        r.simulate_draws()
    bp.set_inputs(ys)
    bp.ws.fill_(0xFF)                                  # stale workspace contents must not matter
    bp.topk()
    torch.cuda.synchronize()
    seen = set()
    for r, y in zip(bp.runs, ys):
        fam = tuple(sorted(r.W.models))
        if fam in seen or r.J < 2:
            continue
        seen.add(fam)
        L = r.L
        yn = y.cpu().numpy()[:, :L]
        xn = r.x.cpu().numpy()[:, :L].astype(np.float64)
        w = r.weights.astype(np.float64)
        oi, od = orc.topk(yn, xn, w, r.k)
        check_topk_sets(r.idx.cpu().numpy(), oi, od, lambda vj, dn: orc.pair_dist(yn, xn, w, vj, dn), L)
    assert len(seen) >= 3


def test_batch_graph_replay(batch):
    from paper_2603_14859_b300 import pipeline
    scans, ys = batch
    bp = pipeline.BatchPipeline(scans, 1)
    bp.set_inputs(ys)
    bp.ws.fill_(0xFF)                                  # stale workspace contents must not matter
    bp.step()
    torch.cuda.synchronize()
    ref = [(r.idx.clone(), r.dist.clone(), r.prob.clone(), r.summ[0].clone()) for r in bp.runs]
    for r in bp.runs:                      # scribble over the outputs, then replay the captured step
        r.idx.fill_(-5)
        r.dist.fill_(-5.0)
    bp.capture()
    for r in bp.runs:
        r.idx.fill_(-5)
    bp.replay()
    bp.replay()
    torch.cuda.synchronize()
    for r, (i, d, p, m) in zip(bp.runs, ref):
        assert torch.equal(r.idx, i) and torch.equal(r.dist, d) and torch.equal(r.prob, p)
        assert torch.equal(torch.nan_to_num(r.summ[0], 7.0), torch.nan_to_num(m, 7.0))


@pytest.mark.parametrize("order_mode", [0, 2])
def test_single_scan_graph_replay(order_mode):
    """One single-scan step (prior draws, simulation, discrepancy + top-k, model selection,
    summaries) captured as a CUDA graph and replayed twice returns, bit for bit, what the eager
    step returns; with the k-d row order forced (mode 2) its level-by-level kernels are in the
    graph too."""
    from paper_2603_14859_b300 import _lib, api, pipeline
    W = S.workload("raclopride_lpntpet", J=700, N_per_model=40000)
    W.k = 50
    y = pipeline.make_y_gpu(W)
    try:
        _lib.check(_lib.lib().abc_debug_order(order_mode))
        run = pipeline.AbcPipeline(W, _lib.ABC_BF16_RESCORE)
        run.ws.fill_(0xFF)                                 # stale workspace contents must not matter
        out = run.step(y)
        torch.cuda.synchronize()
        assert api.topk_status(run.ws)[0] == 0
        fields = ("idx", "dist", "prob", "pref", "mean", "sd", "lo", "hi")
        ref = [torch.nan_to_num(getattr(out, f).clone().float(), 7.0) for f in fields]
        run.capture(y)
        for t in (run.idx, run.dist, run.prob, *run.summ):   # scribble, then replay
            t.fill_(-5)
        run.replay()
        got = run.replay()
        torch.cuda.synchronize()
        assert api.topk_status(run.ws)[0] == 0
    finally:
        _lib.check(_lib.lib().abc_debug_order(0))
    for f, a in zip(fields, ref):
        assert torch.equal(a, torch.nan_to_num(getattr(got, f).float(), 7.0)), f


def test_autotune_choice_and_invariance(batch, tmp_path, monkeypatch):
    from paper_2603_14859_b300 import autotune, pipeline
    monkeypatch.setenv("VPETABC_TUNE_CACHE", str(tmp_path / "tune.json"))
    scans, ys = batch
    bp = pipeline.BatchPipeline(scans, 1)
    for r in bp.runs:
        r.simulate_draws()
    bp.set_inputs(ys)
    bp.ws.fill_(0xFF)                                  # stale workspace contents must not matter
    bp.topk()
    torch.cuda.synchronize()
    ref = [r.idx.clone() for r in bp.runs]
    best = autotune.tune(bp, max_voxels=512, max_draws=20000, reps=1)
    assert best in autotune.CANDIDATES
    assert autotune.tune(bp) == best                   # second call served from the cache
    bp.tuning = best
    bp.topk()
    torch.cuda.synchronize()
    for r, i in zip(bp.runs, ref):
        assert torch.equal(r.idx, i)
    for cand in autotune.CANDIDATES[::5]:               # any tuning gives the same answer
        bp.tuning = cand
        bp.topk()
        torch.cuda.synchronize()
        for r, i in zip(bp.runs, ref):
            assert torch.equal(r.idx, i), cand

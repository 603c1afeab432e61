"""Calibration of the rejection budget on synthetic scans with known truth
(Sec. II-C, the paragraphs on tuning the threshold h, proportion p and draw count n).

For parameter accuracy: over a grid of draw counts n, the mean squared error of
a target parameter's posterior mean against the truth; the MSE-versus-n curve is
U-shaped for a small enough threshold, so a smooth curve (a quadratic in log n)
is fitted and its minimum picks n.  For model selection: over the same kind of
grid, the accuracy of the preferred model and the ROC AUC of the posterior model
probability; the working point is the elbow of the AUC curve.  For activation
detection on the lp-ntPET simulation study's shapes (Sec. IV-A): sensitivity and
specificity of the MRTM / lp-ntPET selection under Gaussian and Poisson noise.

Every ABC step runs in the CUDA library (`pipeline.AbcPipeline`); this module
only loops over the grid and reduces the outputs (the fit, the AUC and the elbow
are small host-side computations).  Run as
`python -m paper_2603_14859_b300.calibrate --mode mse|selection --n 20000,50000,...`.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np

from . import synth as S


# ------------------------------------------------------------------ host-side reductions
def u_curve_minimum(n, mse):
    """Least-squares fit mse ~ a + b u + c u^2 in u = log n; returns (n*, (a, b, c)).
    n* is the fitted minimum when the parabola opens upwards and its vertex lies in
    the grid's range, else the grid point with the smallest observed MSE."""
    n = np.asarray(n, np.float64)
    y = np.asarray(mse, np.float64)
    u = np.log(n)
    if len(n) < 3:
        return float(n[int(np.argmin(y))]), (float("nan"),) * 3
    A = np.stack([np.ones_like(u), u, u * u], axis=1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    a, b, c = (float(v) for v in coef)
    if c > 0:
        uv = -b / (2.0 * c)
        if u.min() <= uv <= u.max():
            return float(math.exp(uv)), (a, b, c)
    return float(n[int(np.argmin(y))]), (a, b, c)


def roc_auc(score, label):
    """Area under the ROC curve of `score` for the binary `label` (Mann-Whitney U
    with average ranks for ties): the probability that a random positive scores
    above a random negative, ties counting one half.  NaN without both classes."""
    s = np.asarray(score, np.float64)
    y = np.asarray(label).astype(bool)
    npos, nneg = int(y.sum()), int((~y).sum())
    if npos == 0 or nneg == 0:
        return float("nan")
    order = np.argsort(s, kind="mergesort")
    ranks = np.empty(len(s), np.float64)
    ss = s[order]
    i = 0
    while i < len(ss):                       # average ranks over runs of equal scores
        j = i
        while j + 1 < len(ss) and ss[j + 1] == ss[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1.0
        i = j + 1
    return float((ranks[y].sum() - npos * (npos + 1) / 2.0) / (npos * nneg))


def elbow(x, y):
    """Index of the elbow of an increasing, flattening curve: after scaling log x
    and y to [0, 1], the point farthest above the chord from the first point to
    the last (the first point when the curve never rises above its chord)."""
    u = np.log(np.asarray(x, np.float64))
    v = np.asarray(y, np.float64)
    if len(u) < 3 or u.max() == u.min() or v.max() == v.min():
        return 0
    un = (u - u.min()) / (u.max() - u.min())
    vn = (v - v.min()) / (v.max() - v.min())
    chord = vn[0] + (vn[-1] - vn[0]) * (un - un[0]) / (un[-1] - un[0])
    gap = vn - chord
    i = int(np.argmax(gap))
    return i if gap[i] > 0 else 0


# ------------------------------------------------------------------ sweeps over the GPU path
@dataclasses.dataclass
class SweepPoint:
    n_per_model: int
    k: int
    seconds: float
    mse: dict | None = None          # model name -> per-column MSE of the posterior mean
    accuracy: float | None = None    # preferred model == true model
    auc: float | None = None         # ROC AUC of P(second model) for the truth "second model"


def _run(name, n, k, p, J, seed, precision, **wkw):
    import torch
    from . import _lib, pipeline
    W = S.workload(name, seed=seed, J=J, N_per_model=n, **wkw)
    W.k = min(W.N, int(k) if k is not None else max(1, int(round(p * W.N))))
    prec = {"fp32": _lib.ABC_FP32, "bf16r": _lib.ABC_BF16_RESCORE, "split": _lib.ABC_SPLIT_DRAWS}[precision]
    run = pipeline.AbcPipeline(W, prec)
    y = pipeline.make_y_gpu(W)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = run.step(y)
    torch.cuda.synchronize()
    return W, out, time.perf_counter() - t0


def mse_sweep(n_grid, k=None, p=None, name="brain_fdg_2tcm", J=4096, seed=None, precision="fp32"):
    """Per n: MSE of every parameter's posterior mean over the voxels whose preferred
    model is their true model (all voxels for a single-model workload)."""
    pts = []
    for n in n_grid:
        W, out, sec = _run(name, int(n), k, p, J, seed, precision)
        mean = out.mean.cpu().numpy().astype(np.float64)
        pref = out.pref.cpu().numpy()
        mse = {}
        for mi, (th, rows) in enumerate(zip(W.truth, W.truth_rows)):
            if len(rows) == 0:
                continue
            m = int(W.truth_model[rows[0]])
            ok = pref[rows] == W.models.index(m)
            P = th.shape[1]
            err = mean[rows][ok, :P] - th[ok].astype(np.float64)
            mse[S.MODEL_NAMES[m]] = (err ** 2).mean(axis=0).tolist() if ok.any() else [float("nan")] * P
        pts.append(SweepPoint(int(n), W.k, sec, mse=mse))
    return pts


def selection_sweep(n_grid, k=None, p=None, name="raclopride_lpntpet", J=8192, seed=None, precision="bf16r"):
    """Per n: accuracy of the preferred model and ROC AUC of the posterior probability
    of the workload's second model (lp-ntPET, or the reversible 2TCM)."""
    pts = []
    for n in n_grid:
        W, out, sec = _run(name, int(n), k, p, J, seed, precision)
        prob = out.prob.cpu().numpy().astype(np.float64)
        pref = out.pref.cpu().numpy()
        truth = np.array([W.models.index(int(m)) for m in W.truth_model])
        pts.append(SweepPoint(int(n), W.k, sec, accuracy=float((pref == truth).mean()),
                              auc=roc_auc(prob[:, 1], truth == 1)))
    return pts


@dataclasses.dataclass
class DetectionPoint:
    noise: str
    level: str
    n_per_model: int
    k: int
    sensitivity: float      # activated voxels whose preferred model is lp-ntPET
    specificity: float      # voxels without activation whose preferred model is MRTM
    auc: float              # ROC AUC of the posterior probability of lp-ntPET
    seconds: float


def detection_sweep(n_grid, k=None, p=None, noises=("gaussian", "poisson"), levels=("low", "high"), J=4000,
                    seed=None, precision="bf16r"):
    """Activation detection on the lp-ntPET simulation study's shapes (Sec. IV-A: 61
    one-minute frames, half the TACs activated, Gaussian and Poisson noise at two
    levels): sensitivity, specificity and AUC of the MRTM / lp-ntPET selection per n."""
    pts = []
    for noise in noises:
        for level in levels:
            for n in n_grid:
                W, out, sec = _run("raclopride_e2", int(n), k, p, J, seed, precision, noise=noise, level=level)
                prob = out.prob.cpu().numpy().astype(np.float64)
                pref = out.pref.cpu().numpy()
                act = W.truth_model == S.LPNTPET
                pts.append(DetectionPoint(noise, level, int(n), W.k, float((pref[act] == 1).mean()),
                                          float((pref[~act] == 0).mean()), roc_auc(prob[:, 1], act), sec))
    return pts


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--mode", choices=["mse", "selection", "detection"], default="mse")
    ap.add_argument("--workload", default=None)
    ap.add_argument("--n", default="10000,20000,50000,100000,200000", help="draws per model, comma-separated")
    ap.add_argument("--k", type=int, default=None, help="accepted draws (fixed)")
    ap.add_argument("--p", type=float, default=None, help="acceptance proportion (k = p n)")
    ap.add_argument("--voxels", type=int, default=None)
    ap.add_argument("--column", type=int, default=0, help="mse mode: target parameter column")
    a = ap.parse_args(argv)
    grid = [int(v) for v in a.n.split(",")]
    if a.k is None and a.p is None:
        a.k = 100
    if a.mode == "mse":
        name = a.workload or "brain_fdg_2tcm"
        pts = mse_sweep(grid, a.k, a.p, name, a.voxels or 4096)
        model = next(iter(pts[0].mse))
        curve = [pt.mse[model][a.column] for pt in pts]
        best, coef = u_curve_minimum(grid, curve)
        res = {"mode": "mse", "workload": name, "model": model, "column": a.column, "n": grid,
               "k": [pt.k for pt in pts], "mse": curve, "fit": coef, "n_best": best,
               "seconds": [pt.seconds for pt in pts]}
    elif a.mode == "detection":
        pts = detection_sweep(grid, a.k, a.p, J=a.voxels or 4000)
        res = {"mode": "detection", "workload": "raclopride_e2", "points": [dataclasses.asdict(pt) for pt in pts]}
    else:
        name = a.workload or "raclopride_lpntpet"
        pts = selection_sweep(grid, a.k, a.p, name, a.voxels or 8192)
        auc = [pt.auc for pt in pts]
        i = elbow(grid, auc)
        res = {"mode": "selection", "workload": name, "n": grid, "k": [pt.k for pt in pts],
               "accuracy": [pt.accuracy for pt in pts], "auc": auc, "n_elbow": grid[i],
               "seconds": [pt.seconds for pt in pts]}
    print(json.dumps(res))
    return res


if __name__ == "__main__":
    main()

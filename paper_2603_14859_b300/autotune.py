"""Autotuner for the batched fused discrepancy + top-k launch.

The fused kernel exposes four launch choices (`abc_tuning`): draws per tile
(64 or 128, which also sets how many CTAs fit on an SM), persistent CTAs per
SM, the draw stride between pilot levels and the pilot safety factor.  None
changes results, only speed.  `tune()` times every candidate on a calibration
view of the batch (each scan truncated to a bounded number of voxels and
draws, without copying), then times the fastest few on the whole batch (the
view misranks choices whose cost depends on the full draw count, such as the
pilot stride) and returns the fastest there; results are cached in a JSON
file keyed by the GPU and a coarse signature of the batch shape.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import statistics

import torch

from . import _lib

CANDIDATES = [
    dict(bn=bn, ctas_per_sm=c, pilot_stride=st, pilot_factor=f)
    for bn, c in [(64, 3), (64, 2), (128, 2), (128, 1)]
    for st in (16, 8)
    for f in (1.5, 2.0)
]


def cache_path() -> str:
    return os.environ.get("VPETABC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "vpetabc", "tuning.json"))


def signature(batch, precision: int) -> str:
    """GPU name + precision + bucketed frames, k, draws and voxel totals."""
    dev = torch.cuda.get_device_name()
    Ls = [r.L for r in batch.runs]
    ks = sorted({r.k for r in batch.runs})
    logN = [round(math.log2(max(r.N, 1))) for r in batch.runs]
    Jtot = sum(r.J for r in batch.runs)
    kblk = "K3" if precision == _lib.ABC_FP32 and max(Ls) > 29 else ("K2" if precision == _lib.ABC_FP32 else "K1")
    return (f"{dev}|p{precision}|{kblk}|n{len(batch.runs)}|L{min(Ls)}-{max(Ls)}|k{ks[0]}-{ks[-1]}"
            f"|N2^{min(logN)}-2^{max(logN)}|J~2^{round(math.log2(max(Jtot, 1)))}")


def _load():
    try:
        return json.load(open(cache_path()))
    except (OSError, ValueError):
        return {}


def _save(d):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    json.dump(d, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, p)


def _calibration_structs(batch, max_voxels: int, max_draws: int):
    """Scan structs over the leading voxels / draws of each scan (no copies)."""
    arr = (_lib.Scan * len(batch.runs))()
    ws_w = []
    for i, (r, y) in enumerate(zip(batch.runs, batch.ys)):
        J = min(r.J, max_voxels)
        N = min(r.N, max_draws)
        k = min(r.k, N)
        w = batch._w[i]
        ws_w.append(w)
        arr[i] = _lib.Scan(y.data_ptr(), J, y.shape[1], r.x.data_ptr(), N, r.x.shape[1], r.L, w.ctypes.data, k,
                           r.idx.data_ptr(), r.dist.data_ptr())
    return arr, ws_w


def _time_call(L, arr, n, precision, t, ws, s, reps):
    times = []
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _lib.check(L.abc_batch_discrepancy_topk(arr, n, precision, ctypes.byref(t), ctypes.c_void_p(ws.data_ptr()),
                                                ws.numel(), ctypes.c_void_p(s.cuda_stream)))
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times[1:])


def tune(batch, precision: int | None = None, max_voxels: int = 4096, max_draws: int = 400_000, reps: int = 2,
         finalists: int = 3, use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick the fastest tuning for `batch` (a pipeline.BatchPipeline with inputs set)."""
    precision = batch.precision if precision is None else precision
    key = signature(batch, precision)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]["tuning"]
    arr, keep = _calibration_structs(batch, max_voxels, max_draws)
    L = _lib.lib()
    n = L.abc_batch_workspace_size(arr, len(batch.runs), precision)
    ws = batch.ws if batch.ws is not None and batch.ws.numel() >= n else torch.empty(n, dtype=torch.uint8,
                                                                                       device="cuda")
    s = torch.cuda.current_stream()
    results = []
    for cand in CANDIDATES:
        t = _lib.Tuning(cand["bn"], cand["ctas_per_sm"], cand["pilot_stride"], cand["pilot_factor"])
        ms = _time_call(L, arr, len(batch.runs), precision, t, ws, s, reps)
        results.append((ms, cand))
        if verbose:
            print(f"  tune {cand}: {ms:.2f} ms")
    results.sort(key=lambda r: r[0])
    # the finalists on the whole batch (its own structs and workspace)
    full = []
    if finalists > 1 and batch._scan_structs is not None and batch.ws is not None:
        for _, cand in results[:finalists]:
            t = _lib.Tuning(cand["bn"], cand["ctas_per_sm"], cand["pilot_stride"], cand["pilot_factor"])
            ms = _time_call(L, batch._scan_structs, len(batch.runs), precision, t, batch.ws, s, 2)
            full.append((ms, cand))
            if verbose:
                print(f"  full batch {cand}: {ms:.2f} ms")
    best = min(full, key=lambda r: r[0]) if full else results[0]
    if use_cache:
        cache[key] = {"tuning": best[1], "ms": best[0], "candidates": [[m, c] for m, c in results],
                      "finalists": [[m, c] for m, c in full]}
        _save(cache)
    return best[1]

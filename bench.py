#!/usr/bin/env python
"""Voxelwise ABC throughput on B300: voxels/s to posterior (and voxel-draw pairs/s).

One step = the whole hot path over one synthetic volume: prior draws and
simulated TACs for every candidate model, tensor-core discrepancy + top-k,
posterior model probabilities and posterior summaries.  Default workload:
the brain lp-ntPET/MRTM model-selection volume (250,000 voxels, 60 one-minute
frames, 1,000,000 draws per model, k = 500), BF16 discrepancy with exact FP32
re-scoring.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision bf16r|fp32|split] [--workload NAME]

Multi-GPU (torchrun): every rank runs its own voxel shard against the same
seeded draws (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "raclopride_lpntpet": "brain lp-ntPET vs MRTM: {J} voxels x ({n} MRTM + {n} lp-ntPET draws), 60 x 1-min frames, k={k}",
    "totalbody_fdg": "total-body FDG 2TCM irr vs rev: {J} voxels x ({n} + {n} draws), 29 frames, k={k}",
    "brain_fdg_2tcm": "2TCM-irr: {J} voxels x {n} draws, 22 frames, k={k}",
    "learned": "learned proposal + local importance-weighted ABC, 2TCM-irr on the total-body FDG volume: {J} voxels x "
               "{M} proposals, 29 frames, k={k}; network trained on {P} simulated pairs; fallback to the global path "
               "({n} 2TCM-irr draws)",
    "batched": "{n} uneven scans: {J} voxels in total (log-uniform 1,000-500,000 per scan), 22-60 frames, 1-3 of "
               "{{2TCM-irr, 2TCM-rev, MRTM}} per scan, 200,000-1,000,000 draws per model, k={k}; one CUDA graph",
}


def _precisions():
    from paper_2603_14859_b300 import _lib
    return {"bf16r": _lib.ABC_BF16_RESCORE, "fp32": _lib.ABC_FP32, "split": _lib.ABC_SPLIT_DRAWS}


PRECISIONS = _precisions()
DTYPES = {"bf16r": "bf16", "fp32": "bf16x3-split (fp32-exact)", "split": "bf16"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16r", choices=["bf16r", "fp32", "split"])
    ap.add_argument("--workload", default="raclopride_lpntpet", choices=sorted(WORKLOADS))
    ap.add_argument("--voxels", type=int, default=None, help="override J (smaller runs)")
    ap.add_argument("--draws", type=int, default=None, help="override draws per model")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="single-scan workloads on N GPUs: every rank a full-size block of the volume (weak) "
                         "or a voxel range of one block (strong)")
    ap.add_argument("--no-fp32-comparator", action="store_true",
                    help="skip the FP32-form sub-record of the fast form's line")
    ap.add_argument("--voxel-scale", type=float, default=1.0, help="batched workload: scale voxel counts")
    ap.add_argument("--draw-scale", type=float, default=1.0, help="batched workload: scale draw counts")
    ap.add_argument("--scans", type=int, default=64, help="batched workload: number of scans")
    ap.add_argument("--proposals", type=int, default=10_000, help="learned workload: proposals per voxel")
    ap.add_argument("--train-pairs", type=int, default=10_000_000, help="learned workload: training pairs")
    ap.add_argument("--sigma-scale", type=float, default=1.0, help="learned workload: proposal widening")
    ap.add_argument("--distance", default="l2", choices=["l2", "l1"],
                    help="single-scan workloads: frame-weighted squared L2 (tensor cores) or L1 (Sec. V; SIMT scan)")
    ap.add_argument("--tuning", default=None,
                    help="single-scan workloads: launch tuning bn,ctas_per_sm,pilot_stride,pilot_factor "
                         "(default: the library's per-precision default)")
    return ap.parse_args()


def kernel_source_sha1() -> str:
    """Hash of the sources the fused kernel is built from; a traffic record taken
    from an older build is not reported."""
    h = hashlib.sha1()
    for f in ("topk.cu", "select.cuh", "tc_ptx.cuh", "topk_internal.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2603_14859_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle baseline
def cpu_baseline(W, seconds_budget=20.0, distance="l2"):
    """The FP64 oracle as it stands, timed on this host on a bounded sample of the
    workload and scaled to voxels/s of the full volume (with the step's distance).  The
    sample is sized from a short probe so that about half of seconds_budget goes to
    simulating draws (shared among the models by their draw counts) and half to ranking
    sampled voxels against them."""
    import oracle
    from paper_2603_14859_b300 import synth as S
    oracle.build()
    cores = oracle.num_threads()
    L = W.L
    # 1. simulation cost per draw, per model
    t_sim = 0.0
    xs = []
    sim_desc = []
    for model, n in zip(W.models, W.n_per_model):
        lo, hi = W.priors(model)
        probe = min(256, n)
        th = oracle.sample_prior(W.prior_seed, model, lo, hi, probe)
        t0 = time.perf_counter()
        oracle.simulate(model, W.ts, W.te, W.inp, th)
        per_draw = max((time.perf_counter() - t0) / probe, 1e-9)
        share = 0.5 * seconds_budget * n / max(W.N, 1)
        ns = int(min(n, 200_000, max(probe, share / per_draw)))
        th = oracle.sample_prior(W.prior_seed, model, lo, hi, ns)
        t0 = time.perf_counter()
        x = oracle.simulate(model, W.ts, W.te, W.inp, th)
        dt = time.perf_counter() - t0
        t_sim += dt / ns * n
        xs.append(x)
        sim_desc.append(f"{ns} {S.MODEL_NAMES[model]} draws")
    xs = np.concatenate(xs)
    # 2. distance + full sort per voxel: sampled voxels against the sampled draws
    rng = np.random.default_rng(0)
    rank = oracle.topk_l1 if distance == "l1" else oracle.topk
    k = min(W.k, len(xs))

    def voxels(nv):
        return (xs[rng.integers(0, len(xs), nv)] * (1 + 0.1 * rng.standard_normal((nv, L)))).astype(np.float32)

    t0 = time.perf_counter()
    rank(voxels(16), xs, W.weights, k)
    per_voxel = max((time.perf_counter() - t0) / 16, 1e-9)
    nv = int(min(4096, max(16, 0.5 * seconds_budget / per_voxel)))
    y = voxels(nv)
    t0 = time.perf_counter()
    rank(y, xs, W.weights, k)
    dt = time.perf_counter() - t0
    per_pair = dt / (nv * len(xs))
    t_topk = per_pair * W.J * W.N * math.log(W.N) / math.log(len(xs))   # n log n sort
    total = t_sim + t_topk
    return {"value": W.J / total, "unit": "voxels/s", "cores": cores, "kind": "oracle",
            "sample": (f"simulation timed on {', '.join(sim_desc)}; {distance} distance+sort timed on {nv} voxels x "
                       f"{len(xs)} draws; scaled to {W.J} voxels x {W.N} draws (sort as n log n)"),
            "pairs_per_s": W.J * W.N / total}


# ------------------------------------------------------------------ batched uneven scans
def run_batched(args, world, rank, local):
    """Many scans per step: prior draws and simulation per scan, one batched
    discrepancy + top-k (persistent fused kernel, autotuned launch), model
    selection and summaries per scan, the whole step replayed from a CUDA graph."""
    import torch
    from paper_2603_14859_b300 import _lib, api, autotune, pipeline
    from paper_2603_14859_b300 import synth as S
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    prec = PRECISIONS[args.precision]
    plan = S.scan_plan(seed=1004 + 1000 * rank, n_scans=args.scans, voxel_scale=args.voxel_scale,
                       draw_scale=args.draw_scale)
    scans = [S.scan_workload(p) for p in plan]
    bp = pipeline.BatchPipeline(scans, prec)
    ys = [pipeline.make_y_gpu(W) for W in scans]
    bp.set_inputs(ys)
    for r in bp.runs:
        r.simulate_draws()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bp.tuning = autotune.tune(bp)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    prof = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in prof:
        e.record(stream)
    torch.cuda.synchronize()
    api.profile_events(*prof)
    l0 = api.launch_info()[2]
    bp.capture()                                   # one eager warm-up step, then the captured step
    launches_per_step = (api.launch_info()[2] - l0) // 2
    for _ in range(args.warmup):
        bp.replay()
    torch.cuda.synchronize()
    st = api.topk_status(bp.ws)
    K = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    tc = []
    for _ in range(K):
        bp.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        tc.append(prof[0].elapsed_time(prof[1]))
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / K
    api.profile_events(None, None)
    # end to end: pinned host TACs in, model probabilities and summaries out, around each replay
    y_host = [y.cpu().pin_memory() for y in ys]
    outs = [(r.prob, r.pref, *r.summ) for r in bp.runs]
    outs_host = [[torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in grp] for grp in outs]
    h2d = sum(y.numel() * y.element_size() for y in y_host)
    d2h = sum(o.numel() * o.element_size() for grp in outs_host for o in grp)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ke = max(1, min(K, 3))
    f0.record(stream)
    for _ in range(Ke):
        for yd, yh in zip(ys, y_host):
            yd.copy_(yh, non_blocking=True)
        bp.replay()
        for grp_h, grp_d in zip(outs_host, outs):
            for h, d in zip(grp_h, grp_d):
                h.copy_(d, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / Ke
    t = torch.tensor([ms, statistics.mean(tc), e2e_ms], device="cuda", dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, tc_ms, e2e_ms = (float(v) for v in t)
    if rank != 0:
        dist.destroy_process_group()
        return
    J = sum(W.J for W in scans)
    pairs = sum(W.J * W.N for W in scans)
    flops = sum(2.0 * W.L * W.J * W.N for W in scans)
    kept, total_tiles = api.topk_work(bp.ws)
    cols = {0: 3, 1: 2, 2: 2}[prec]
    kp = max(-(-(cols * W.L + 3) // 64) * 64 for W in scans)
    executed = (2.0 * 128 * 64 * kp * kept) if total_tiles else flops * kp / max(W.L for W in scans)   # 64-draw tiles
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops_sustained", 1400.0)
    achieved = executed / (tc_ms / 1000.0) / 1e12
    cfg = {"workload": WORKLOADS["batched"].format(n=len(scans), J=J, k=scans[0].k), "scans": len(scans),
           "voxels_per_gpu": J, "pairs_per_gpu": pairs, "voxel_scale": args.voxel_scale,
           "draw_scale": args.draw_scale, "precision": args.precision, "tuning": bp.tuning,
           "autotune_s": tune_s, "l2": "inputs larger than L2",
           "parallelism": f"voxel shards x{args.gpus}" if args.gpus > 1 else "single GPU"}
    line = {
        "metric": "voxels/s to posterior", "value": J * world / (ms / 1000.0), "unit": "voxels/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic", "config": cfg, "pairs_per_s": pairs * world / (ms / 1000.0),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_tc_topk main pass (all scans, one persistent launch)",
                     "kernel_ms": tc_ms, "executed_flops_per_launch": executed,
                     "executed": "bf16 MMA flops of the draw tiles processed (128 x 64 x Kp x 2 per 64-draw tile)",
                     "tiles_processed": kept, "tiles_without_skipping": total_tiles,
                     "algorithmic_flops_per_launch": flops,
                     "algorithmic_equivalent_tflops": flops / (tc_ms / 1000.0) / 1e12,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"},
        "e2e": {"value": J * world / (e2e_ms / 1000.0), "unit": "voxels/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * K,
        "clocks": clk,
        "topk_status": {"error": st[0], "exact_scan_voxels": st[1], "tie_overflow_voxels": st[2],
                        "uncertified_voxels": st[3],
                        "diagnostics": list(st[4:8])},
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ learned proposal + local ABC
# Algorithmic work of one local proposal evaluated directly: per frame, cubic interpolation 8, model
# combination 6, residual and weighted square 4 flops (the kernel's quadratic form avoids most of it).
LOCAL_FLOPS_PER_FRAME = 18
# Thread instructions the local ABC kernel issues per proposal (ncu smsp__inst_executed x 32 / proposals,
# measured on the 40,000-voxel learned case).  The kernel is issue-bound, so its roofline is instruction
# issue against the SIMT issue peak.
LOCAL_INST_PER_PROPOSAL = 523.0


def cpu_baseline_learned(W, M, k, model_params, D, H, seconds_budget=20.0):
    """The FP64 oracle as it stands on a bounded sample of the learned workload:
    network forward, truncated-normal proposals, simulation of every proposal and
    the importance-weighted local ABC, for a few voxels; scaled to the volume."""
    import oracle
    from paper_2603_14859_b300 import synth as S
    oracle.build()
    cores = oracle.num_threads()
    lo, hi = (np.asarray(a, np.float64) for a in S.PRIORS[S.TCM2_IRR])
    w = W.weights.astype(np.float64)
    rng = np.random.default_rng(0)
    ys = []
    for th, rows in zip(W.truth, W.truth_rows):
        if W.truth_model[rows[0]] == S.TCM2_IRR:
            x = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.input_for(S.TCM2_IRR), th[:2])
            ys = (x * (1 + 0.1 * rng.standard_normal(x.shape))).astype(np.float32)
    prm = np.asarray(model_params, np.float64)
    t0 = time.perf_counter()
    nv = 0
    for yv in ys:
        s = math.sqrt(float((w * yv.astype(np.float64) ** 2).sum()))
        feat = np.concatenate([yv / s, [math.log(s) / 10]])[None, :]
        out = oracle.mlp_forward(prm, D, H, 8, feat)[0]
        mu = np.clip(out[0::2], -3, 4)
        sg = np.exp(np.clip(out[1::2], -7, 2))
        uni = rng.random((M, 4))
        u = np.array([[oracle.truncnorm01(mu[p], sg[p], uni[i, p]) for p in range(4)] for i in range(M)])
        th = (lo + (hi - lo) * u).astype(np.float32)
        x = oracle.simulate(S.TCM2_IRR, W.ts, W.te, W.input_for(S.TCM2_IRR), th)
        oracle.local_abc(u, mu, sg, x, yv, w, k, lo, hi)
        nv += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    dt = (time.perf_counter() - t0) / nv
    return {"value": 1.0 / dt, "unit": "voxels/s", "cores": cores, "kind": "oracle",
            "sample": f"{nv} voxels end to end (FP64 network, {M} truncated-normal proposals, FP64 simulation of "
                      f"each, weighted local ABC); scaled per voxel (fallback voxels not included)"}


def run_learned_bench(args, world, rank, local):
    """One step = network features + forward over every voxel, local ABC with M
    proposals per voxel, and the global path for the voxels that fall back."""
    import torch
    from paper_2603_14859_b300 import api, learned
    from paper_2603_14859_b300 import pipeline
    from paper_2603_14859_b300 import synth as S
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    W = S.workload("totalbody_fdg", seed=None if rank == 0 else 5000 + rank, J=args.voxels)
    M, k = args.proposals, W.k
    model = learned.LearnedLocalAbc(W.ts, W.te, W.input_for(S.TCM2_IRR), W.half_life)
    tl = model.train(n_pairs=args.train_pairs)
    n_glob = args.draws or 1_000_000
    g = learned.GlobalIrr(model, N=n_glob, k=k)
    y = pipeline.make_y_gpu(W)
    rel = g.calibrate(y[:2048].contiguous())
    g.reserve(W.J)
    stream = torch.cuda.current_stream()
    J = W.J
    outs = dict(mean=torch.empty((J, 5), device="cuda"), sd=torch.empty((J, 5), device="cuda"),
                lo=torch.empty((J, 5), device="cuda"), hi=torch.empty((J, 5), device="cuda"),
                ess=torch.empty(J, device="cuda"), dmed=torch.empty(J, device="cuda"),
                ynorm=torch.empty(J, device="cuda"))
    prop = torch.empty((J, 8), device="cuda")
    ev_local = []

    def step(yd, rec=None):
        model.propose(yd, out=prop)
        if rec is not None:
            rec[0].record(stream)
        model.local(yd, prop, M=M, k=k, sigma_scale=args.sigma_scale, out=outs)
        if rec is not None:
            rec[1].record(stream)
        return learned.fallback_to_global(outs, yd, k, g, rel)[1]

    for _ in range(args.warmup):
        step(y)
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in ev:
        a.record(stream)
        b.record(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = api.launch_info()[2]
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    nfb = [step(y, ev[i]) for i in range(K)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = api.launch_info()[2] - l0
    ms = e0.elapsed_time(e1) / K
    local_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # end to end: pinned host TACs in, posterior summaries out
    y_host = y.cpu().pin_memory()
    y_dev = torch.empty_like(y)
    outs_host = [torch.empty(outs[key].shape).pin_memory() for key in ("mean", "sd", "lo", "hi")]
    Ke = max(1, min(K, 3))
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(Ke):
        y_dev.copy_(y_host, non_blocking=True)
        step(y_dev)
        for h, key in zip(outs_host, ("mean", "sd", "lo", "hi")):
            h.copy_(outs[key], non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / Ke
    # accuracy against the global path on a voxel sample (outside the timed region)
    sub = y[:4096].contiguous()
    ref = g.run(sub)["mean"].cpu().numpy()
    got = outs["mean"][:4096].cpu().numpy()
    g2 = learned.GlobalIrr(model, N=n_glob, k=k, seed=4321)
    ref2 = g2.run(sub)["mean"].cpu().numpy()
    rel_l2 = lambda a, b: [float(np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c])) for c in range(5)]
    # the global path alone over the whole volume (no network), FP32 and fast exact forms, same
    # draws: the comparators of the learned form (outside the timed region)
    comparators = {}
    if not args.no_fp32_comparator:
        for name, prec in (("global_fp32", PRECISIONS["fp32"]), ("global_bf16r", PRECISIONS["bf16r"])):
            gp = g if prec == g.precision else learned.GlobalIrr(model, N=n_glob, k=k, seed=1234, precision=prec)
            gp.run(y)
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nrep = 2
            c0.record(stream)
            for _ in range(nrep):
                gp.run(y)
            c1.record(stream)
            torch.cuda.synchronize()
            gms = c0.elapsed_time(c1) / nrep
            comparators[name] = {"ms_per_step": gms, "voxels_per_s": J / (gms / 1000.0), "draws": n_glob,
                                 "steps": nrep}
            if gp is not g:
                del gp
                torch.cuda.empty_cache()
    t = torch.tensor([ms, local_ms, e2e_ms], device="cuda", dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, local_ms, e2e_ms = (float(v) for v in t)
    if rank != 0:
        dist.destroy_process_group()
        return
    flops = float(LOCAL_FLOPS_PER_FRAME) * W.L * J * M
    inst = LOCAL_INST_PER_PROPOSAL * J * M
    achieved = inst / (local_ms / 1000.0) / 1e12
    sm_mhz = clk["sm_mhz"] if clk else 2032.0
    peak = 148 * 4 * 32 * sm_mhz * 1e6 / 1e12
    cfg = {"workload": WORKLOADS["learned"].format(J=J, M=M, k=k, P=tl.pairs, n=n_glob), "voxels_per_gpu": J,
           "proposals_per_voxel": M, "frames": W.L, "k": k, "sigma_scale": args.sigma_scale,
           "training": {"pairs": tl.pairs, "steps": tl.steps, "seconds": tl.seconds,
                        "pairs_per_s": tl.pairs / tl.seconds, "final_loss": tl.losses[-1][1]},
           "fallback": {"rule": "ESS < k/4 or median accepted distance > calibrated relative threshold",
                        "rel_threshold": rel, "voxels_per_step": statistics.mean(nfb)},
           "accuracy_vs_global": {"columns": ["K1", "k2", "k3", "Vb", "Ki"], "sample_voxels": 4096,
                                  "rel_l2_learned": rel_l2(got, ref), "rel_l2_global_reseeded": rel_l2(ref2, ref)},
           "l2": "inputs larger than L2", "parallelism": f"voxel shards x{args.gpus}" if args.gpus > 1 else "single GPU"}
    if comparators:
        cfg["global_comparators"] = comparators
    line = {
        "metric": "voxels/s to posterior", "value": J * world / (ms / 1000.0), "unit": "voxels/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (network weights bf16)", "data": "synthetic", "config": cfg,
        "pairs_per_s": J * M * world / (ms / 1000.0),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T thread-instructions/s",
                     "frac": achieved / peak,
                     "traffic": None, "kernel": "k_local_abc (proposals, TACs, distances, selection, summaries)",
                     "kernel_ms": local_ms, "instructions_per_launch": inst,
                     "instructions_per_proposal": LOCAL_INST_PER_PROPOSAL,
                     "peak_source": "SIMT issue: 148 SMs x 4 schedulers x 32 lanes x median SM clock under load",
                     "algorithmic_flops_per_launch": flops,
                     "algorithmic_equivalent_tflops": flops / (local_ms / 1000.0) / 1e12,
                     "algorithmic_note": "direct evaluation: 18 flop per frame per proposal, against the FP32 lanes "
                                         "(148 x 128 x 2 x clock)"},
        "e2e": {"value": J * world / (e2e_ms / 1000.0), "unit": "voxels/s",
                "h2d_bytes_per_step": y_host.numel() * 4, "d2h_bytes_per_step": sum(o.numel() * 4 for o in outs_host)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_learned(W, M, k, model.params.cpu().numpy(), model.D, model.H)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ main
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2603_14859_b300 import synth as S

    from paper_2603_14859_b300 import sharding

    def make_workload(r):
        return sharding.rank_workload(args.workload, r, world, J=args.voxels, N_per_model=args.draws,
                                      scaling=args.scaling)

    if args.workload == "batched":
        return run_batched(args, world, rank, local)
    if args.workload == "learned":
        if args.impl == "ours":
            return run_learned_bench(args, world, rank, local)
        if rank != 0:
            return
        # reference arm: the FP64 oracle's learned path on the host cores (network parameters
        # drawn at random: the oracle's cost does not depend on their values)
        W = S.workload("totalbody_fdg", J=args.voxels)
        D, H = W.L + 1, 256
        prm = np.random.default_rng(0).normal(0.0, 0.05, H * D + H + H * H + H + 8 * H + 8)
        vals, cb = [], None
        for _ in range(args.warmup + args.steps):
            cb = cpu_baseline_learned(W, args.proposals, W.k, prm, D, H, seconds_budget=10.0)
            vals.append(cb["value"])
        v = statistics.median(vals[args.warmup:]) if args.steps else vals[-1]
        cb["value"] = v
        cfg = {"workload": WORKLOADS["learned"].format(J=W.J, M=args.proposals, k=W.k, P=args.train_pairs,
                                                       n=args.draws or 1_000_000), "voxels_per_gpu": W.J}
        print(json.dumps({"impl": "reference", "metric": "voxels/s to posterior", "value": v, "unit": "voxels/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1000.0 * W.J / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                          "cpu_baseline": cb, "e2e": {"value": v, "unit": "voxels/s", "h2d_bytes_per_step": 0,
                                                      "d2h_bytes_per_step": 0}}))
        return
    W = make_workload(rank)
    cfg = {"workload": WORKLOADS[args.workload].format(J=W.J, n=W.n_per_model[0], k=W.k),
           "voxels_per_gpu": W.J, "draws": W.N, "frames": W.L, "k": W.k,
           "precision": args.precision, "l2": "inputs larger than L2 (draw operands + candidate lists > 126 MB)",
           "parallelism": (f"disjoint voxel ranges of one volume x{args.gpus} ({args.scaling} scaling)"
                           if args.gpus > 1 else "single GPU")}
    if args.tuning and args.impl != "reference":
        from paper_2603_14859_b300 import api as _api
        bn, cps, st, fac = args.tuning.split(",")
        _api.set_default_tuning(int(bn), int(cps), int(st), float(fac))
        cfg["tuning"] = {"bn": int(bn), "ctas_per_sm": int(cps), "pilot_stride": int(st), "pilot_factor": float(fac)}

    if args.impl == "reference":
        if rank != 0:
            return
        # the reference arm is the FP64 oracle on the host cores
        vals = []
        cb = None
        for _ in range(args.warmup + args.steps):
            cb = cpu_baseline(W, seconds_budget=10.0, distance=args.distance)
            vals.append(cb["value"])
        v = statistics.median(vals[args.warmup:]) if args.steps else vals[-1]
        cb["value"] = v
        print(json.dumps({"impl": "reference", "metric": "voxels/s to posterior", "value": v, "unit": "voxels/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1000.0 * W.J / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                          "cpu_baseline": cb, "e2e": {"value": v, "unit": "voxels/s", "h2d_bytes_per_step": 0,
                                                      "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2603_14859_b300 import _lib, api, pipeline
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    prec = PRECISIONS[args.precision]
    l1 = args.distance == "l1"
    run = pipeline.AbcPipeline(W, prec, distance=args.distance)
    y = pipeline.make_y_gpu(W)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        run.step(y)
    torch.cuda.synchronize()
    st = api.topk_status(run.ws) if not l1 else [0, 0, api.l1_status(run.ws, W.J, W.k), 0, 0, 0, 0, 0]
    K = args.steps
    # the squared-L2 step runs as one CUDA graph (its launches counted once, at capture); the
    # fused main pass is bracketed by events recorded inside the graph, read after each replay.
    # The L1 step runs eagerly, its launches counted by the library.
    use_graph = not l1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if use_graph:
        prof = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        for e in prof:
            e.record(stream)
        torch.cuda.synchronize()
        api.profile_events(*prof)
        l0 = api.launch_info()[2]
        run.capture(y)                     # one eager step, then the captured step
        launches_per_step = (api.launch_info()[2] - l0) // 2
        api.profile_events(None, None)
        for _ in range(2):
            run.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        e0.record(stream)
        tcs = []
        for i in range(K):
            run.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            tcs.append(prof[0].elapsed_time(prof[1]))
        launches = launches_per_step * K
        barrier()
        ms = e0.elapsed_time(e1) / K
        tc_ms = statistics.mean(tcs)
        cfg["step_launch"] = f"one CUDA graph replay per step ({launches_per_step} kernels)"
    else:
        launches0 = api.launch_info()[2]
        # timed region (device time on the launching stream)
        clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        e0.record(stream)
        for i in range(K):
            run.step(y)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = api.launch_info()[2] - launches0
        barrier()
        ms = e0.elapsed_time(e1) / K
        # the L1 scan + final selection, timed alone on the same inputs
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        api.discrepancy_topk_l1(y, run.x, W.L, run.weights, W.k, run.ws, run.idx, run.dist, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        tc_ms = a.elapsed_time(b)
    clk = clocks.stop()
    ms, tc_ms = sharding.max_over_ranks([ms, tc_ms], dist, device="cuda")
    voxels_all = int(round(sharding.sum_over_ranks(W.J, dist, device="cuda")))

    # end to end through the public API with host buffers: pinned TACs into the step's input
    # buffer, the step (graph replay, or the eager L1 step), model probabilities and summaries out
    y_host = y.cpu().pin_memory()
    outs_host = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in [run.prob, run.pref] + run.summ]
    h2d = y_host.numel() * y_host.element_size()
    d2h = sum(o.numel() * o.element_size() for o in outs_host)
    Ke = max(1, min(K, 3))
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(Ke):
        y.copy_(y_host, non_blocking=True)
        out = run.replay() if use_graph else run.step(y)
        for h, d in zip(outs_host, [out.prob, out.pref, out.mean, out.sd, out.lo, out.hi]):
            h.copy_(d, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / Ke
    e2e_ms = sharding.max_over_ranks([e2e_ms], dist, device="cuda")[0]
    resp = response_band_timing(W, run, stream, clk) if rank == 0 else None

    if rank != 0:
        dist.destroy_process_group()
        return
    n_gpu = world
    voxels = voxels_all
    value = voxels / (ms / 1000.0)
    flops = 2.0 * W.L * W.J * W.N
    kept, total_tiles = api.topk_work(run.ws) if not l1 else (0, 0)
    kp = -(-(({0: 3, 1: 2, 2: 2}[prec]) * W.L + 3) // 64) * 64
    executed = (2.0 * 128 * 64 * kp * kept) if total_tiles else 2.0 * kp * W.J * W.N   # kept: 64-draw tiles
    achieved = executed / (tc_ms / 1000.0) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops_sustained", 1400.0)
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        h = kernel_source_sha1()
        rec = json.load(open(tp)).get(f"{args.workload}/{args.precision}")
        if rec and rec.get("source_sha1") == h:
            traffic = rec["bytes_per_launch"]
    line = {
        "metric": "voxels/s to posterior", "value": value, "unit": "voxels/s", "n_gpus": n_gpu, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": args.scaling,
        "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic", "config": cfg,
        "pairs_per_s": voxels * W.N / (ms / 1000.0),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_tc_topk main pass (fused discrepancy + top-k filter)", "kernel_ms": tc_ms,
                     "executed_flops_per_launch": executed,
                     "executed": "bf16 MMA flops of the draw tiles processed (128 x 64 x Kp x 2 per 64-draw tile)",
                     "tiles_processed": kept, "tiles_without_skipping": total_tiles,
                     "algorithmic_flops_per_launch": flops,
                     "algorithmic_equivalent_tflops": flops / (tc_ms / 1000.0) / 1e12,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"},
        "e2e": {"value": voxels / (e2e_ms / 1000.0), "unit": "voxels/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "topk_status": {"error": st[0], "exact_scan_voxels": st[1], "tie_overflow_voxels": st[2], "uncertified_voxels": st[3],
                        "diagnostics": list(st[4:8])},
    }
    if l1:
        sm_mhz = clk["sm_mhz"] if clk else 2032.0
        lane_peak = 148 * 128 * sm_mhz * 1e6 / 1e12
        inst = 2.0 * W.L * W.J * W.N            # per (voxel, draw, frame): a subtraction and an fma
        line["dtype"] = "f32"
        line["config"]["distance"] = "frame-weighted L1 (Sec. V)"
        line["roofline"] = {"bound": "alu", "achieved": inst / (tc_ms / 1000.0) / 1e12, "peak": lane_peak,
                            "unit": "T FP32 lane-instructions/s", "frac": inst / (tc_ms / 1000.0) / 1e12 / lane_peak,
                            "traffic": None, "kernel": "k_l1_scan + k_l1_final (SIMT L1 scan, lists, selection)",
                            "kernel_ms": tc_ms, "instructions_per_launch": inst,
                            "peak_source": "FP32 lanes: 148 SMs x 128 x median SM clock under load"}
        line["topk_status"] = {"tie_overflow_voxels": st[2]}
    if resp is not None:
        line["response_band"] = resp
    if not l1 and prec != _lib.ABC_FP32 and rank == 0:
        if args.no_fp32_comparator or W.J > 1_000_000:
            line["stated_error"] = {"accepted_sets": "exact fp32 top-k, certified per voxel (uncertified nets "
                                                     "re-collected by the rescue pass or the exact scan); parity "
                                                     "against the FP64 oracle at full size in "
                                                     "tests/test_gpu_fullsize.py"}
        else:
            line.update(fp32_comparator(W, run, y, stream, peak, K, args.warmup))
    if n_gpu == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W, distance=args.distance)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def fp32_comparator(W, run, y, stream, peak, K, warmup):
    """The same step with the ABC_FP32 form (three bf16 products per term), timed in the
    same run, and the fast form's error against it: both return the exact fp32 top-k, so
    the accepted sets may differ only where fp32 distances tie; the summaries are compared
    over every voxel."""
    import torch
    from paper_2603_14859_b300 import _lib, api, pipeline
    out = run.step(y)
    torch.cuda.synchronize()
    fast = [t.clone() for t in (out.idx, out.prob, out.pref, out.mean, out.sd, out.lo, out.hi)]
    rf = pipeline.AbcPipeline(W, _lib.ABC_FP32)
    for _ in range(max(2, warmup)):
        rf.step(y)
    torch.cuda.synchronize()
    Kf = max(1, min(K, 3))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Kf)]
    for a, b in ev:
        a.record(stream)
        b.record(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(Kf):
        api.profile_events(*ev[i])
        of = rf.step(y)
    e1.record(stream)
    torch.cuda.synchronize()
    api.profile_events(None, None)
    ms = e0.elapsed_time(e1) / Kf
    tc_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    st = api.topk_status(rf.ws)
    kept, total_tiles = api.topk_work(rf.ws)
    kp = -(-(3 * W.L + 3) // 64) * 64
    executed = (2.0 * 128 * 64 * kp * kept) if total_tiles else 2.0 * kp * W.J * W.N
    same = (torch.sort(fast[0], 1).values == torch.sort(of.idx, 1).values).all(1)
    rel = {}
    for name, a, b in zip(("mean", "sd", "lo", "hi"), fast[3:], (of.mean, of.sd, of.lo, of.hi)):
        m = ~torch.isnan(b)
        d = torch.where(m, (a - b).abs() / b.abs().clamp_min(1e-12), torch.zeros_like(b))
        rel[name] = float(d.max())
    rec = {
        "fp32_exact": {"ms_per_step": ms, "value": W.J / (ms / 1000.0), "unit": "voxels/s", "steps": Kf,
                       "kernel_ms": tc_ms, "executed_tflops": executed / (tc_ms / 1000.0) / 1e12,
                       "frac": executed / (tc_ms / 1000.0) / 1e12 / peak, "exact_scan_voxels": st[1],
                       "dtype": DTYPES["fp32"]},
        "stated_error": {
            "accepted_sets": "exact fp32 top-k, certified per voxel (uncertified nets re-collected by the rescue "
                             "pass or the exact scan); parity against the FP64 oracle at full size in "
                             "tests/test_gpu_fullsize.py",
            "voxels_with_sets_equal_to_fp32_form": int(same.sum()), "voxels": W.J,
            "max_rel_diff_vs_fp32_form": rel,
            "model_prob_max_abs_diff_vs_fp32_form": float((fast[1] - of.prob).abs().max()),
            "preferred_model_differs": int((fast[2] != of.pref).sum())},
    }
    del rf
    torch.cuda.empty_cache()
    return rec


# thread instructions per response evaluation of k_response_cri (evaluation, compensated
# mean and the histogram order statistics over the accepted lp-ntPET draws), measured by
# ncu (smsp__thread_inst_executed.sum) on the brain lp-ntPET workload
RESP_INST_PER_RESPONSE = 205.8


def response_band_timing(W, run, stream, clk, reps=3):
    """Posterior band of the lp-ntPET response function at the frame mid-times for
    every voxel of the last step (an extra output, outside the timed step)."""
    import torch
    from paper_2603_14859_b300 import api
    from paper_2603_14859_b300 import synth as S
    if S.LPNTPET not in W.models:
        return None
    mi = list(W.models).index(S.LPNTPET)
    first, last = int(run.offsets[mi]), int(run.offsets[mi + 1])
    tmid = ((np.asarray(W.ts) + np.asarray(W.te)) / 2.0).astype(np.float32)
    out = api.response_cri(run.theta, first, last, tmid, run.idx, stream=stream)
    api.response_cri(run.theta, first, last, tmid, run.idx, out=out, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        api.response_cri(run.theta, first, last, tmid, run.idx, out=out, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    r_ms = a.elapsed_time(b) / reps
    n_acc = int(((run.idx >= first) & (run.idx < last)).sum().item())
    n_resp = n_acc * len(tmid)
    rec = {"kernel": "k_response_cri", "kernel_ms": r_ms, "voxels": W.J, "times": len(tmid),
           "accepted_lpntpet_draws": n_acc, "responses_per_s": n_resp / (r_ms / 1000.0),
           "voxels_per_s": W.J / (r_ms / 1000.0)}
    if RESP_INST_PER_RESPONSE is not None:
        sm_mhz = clk["sm_mhz"] if clk else 2032.0
        peak = 148 * 4 * 32 * sm_mhz * 1e6 / 1e12
        achieved = RESP_INST_PER_RESPONSE * n_resp / (r_ms / 1000.0) / 1e12
        rec["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T thread-instructions/s",
                           "frac": achieved / peak, "instructions_per_response": RESP_INST_PER_RESPONSE,
                           "peak_source": "SIMT issue: 148 SMs x 4 schedulers x 32 lanes x median SM clock"}
    return rec


if __name__ == "__main__":
    main()

"""One pass of the voxelwise ABC hot path on the GPU (Algorithm 1).

    run = AbcPipeline(workload, precision)        # allocates device buffers once
    out = run.step(y_dev)                         # prior -> simulate -> top-k -> select -> summarise

Every stage is a call into the CUDA library; this module only allocates
device memory and sequences the calls on one stream.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _lib, api
from . import synth as S

HAS_KI = {S.TCM2_IRR: 1, S.TCM2_REV: 1, S.MRTM: 0, S.LPNTPET: 0}


@dataclasses.dataclass
class StepOutput:
    idx: torch.Tensor
    dist: torch.Tensor
    prob: torch.Tensor
    pref: torch.Tensor
    mean: torch.Tensor
    sd: torch.Tensor
    lo: torch.Tensor
    hi: torch.Tensor


class AbcPipeline:
    def __init__(self, W: S.Workload, precision: int | None = None, ldtheta: int = 8, own_workspace: bool = True,
                 distance: str = "l2"):
        self.W = W
        self.precision = (_lib.ABC_FP32 if W.precision == "fp32" else _lib.ABC_BF16_RESCORE) if precision is None \
            else precision
        self.L = W.L
        self.ldx = ((self.L + 3) // 4) * 4
        self.N = W.N
        self.J = W.J
        self.k = W.k
        self.offsets = W.model_offsets()
        self.nparams = [len(S.PARAM_NAMES[m]) for m in W.models]
        self.has_ki = [HAS_KI[m] for m in W.models]
        dev = "cuda"
        self.theta = torch.zeros((self.N, ldtheta), dtype=torch.float32, device=dev)
        self.x = torch.zeros((self.N, self.ldx), dtype=torch.float32, device=dev)
        self.distance = distance
        if distance == "l1":      # Sec. V's L1 distance: SIMT scan, its own candidate-list workspace
            self.ws = torch.empty(api.l1_workspace_size(self.J, self.k), dtype=torch.uint8, device="cuda")
        else:
            self.ws = api.alloc_workspace(self.J, self.N, self.L, self.k, self.precision) if own_workspace else None
        self.idx = torch.empty((self.J, self.k), dtype=torch.int32, device=dev)
        self.dist = torch.empty((self.J, self.k), dtype=torch.float32, device=dev)
        M = len(W.models)
        self.prob = torch.empty((self.J, M), dtype=torch.float32, device=dev)
        self.pref = torch.empty(self.J, dtype=torch.int8, device=dev)
        nc = max(self.nparams) + 1
        self.summ = [torch.empty((self.J, nc), dtype=torch.float32, device=dev) for _ in range(4)]
        self.weights = W.weights.astype(np.float32)
        self.graph = None

    def simulate_draws(self, stream=None):
        """Algorithm 1, steps 1-3: prior draws and their TACs for every model."""
        W = self.W
        for m, model in enumerate(W.models):
            a, b = self.offsets[m], self.offsets[m + 1]
            lo, hi = W.priors(model)
            api.sample_prior(W.prior_seed, model, lo, hi, b - a, 0, out=self.theta[a:b], stream=stream)
            api.simulate(model, W.ts, W.te, W.input_for(model), self.theta[a:b], out=self.x[a:b], stream=stream)

    def select(self, y, stream=None):
        """Algorithm 1, steps 4-5 plus model probabilities and summaries."""
        if self.distance == "l1":
            api.discrepancy_topk_l1(y, self.x, self.L, self.weights, self.k, self.ws, self.idx, self.dist, stream=stream)
        else:
            api.discrepancy_topk(y, self.x, self.L, self.weights, self.k, self.precision, self.ws, self.idx,
                                 self.dist, stream=stream)
        api.model_select(self.idx, self.offsets, self.prob, self.pref, stream=stream)
        pref = self.pref if len(self.W.models) > 1 else None
        api.summarize(self.theta, self.offsets, self.nparams, self.has_ki, [0, 1, 2], self.idx, pref, out=self.summ,
                      stream=stream)

    def step(self, y, stream=None) -> StepOutput:
        self.simulate_draws(stream)
        self.select(y, stream)
        return self.outputs()

    def outputs(self) -> StepOutput:
        return StepOutput(self.idx, self.dist, self.prob, self.pref, *self.summ)

    def capture(self, y):
        """Record one step on the voxel TACs in `y` into a CUDA graph, after one eager
        warm-up step on a side stream.  The graph reads `y` in place: refill that buffer
        between replays.  The squared-L2 path only (the L1 call reads a status word back)."""
        if self.distance != "l2":
            raise ValueError("capture: the L1 path is not captured")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step(y)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step(y)
        torch.cuda.synchronize()

    def replay(self) -> StepOutput:
        self.graph.replay()
        return self.outputs()


def truth_groups(W: S.Workload):
    """(model, voxel rows, truth parameters) for each group of ground-truth voxels."""
    for th, rows in zip(W.truth, W.truth_rows):
        if len(rows):
            yield int(W.truth_model[rows[0]]), rows, th


def make_y_gpu(W: S.Workload, stream=None) -> torch.Tensor:
    """Measured voxel TACs: GPU-simulated truth curves plus the seeded noise model."""
    L = W.L
    ldy = ((L + 3) // 4) * 4
    x_clean = np.zeros((W.J, L), np.float64)
    for model, rows, th in truth_groups(W):
        xc = api.simulate(model, W.ts, W.te, W.input_for(model), torch.from_numpy(np.ascontiguousarray(th)).cuda(),
                          stream=stream)
        x_clean[rows] = xc[:, :L].cpu().numpy()
    if W.noise == "poisson":
        y = S.add_noise_poisson(x_clean, S.poisson_scale(x_clean, W.noise_q), W.noise_seed)
    else:
        y = S.add_noise(x_clean, W.ts, W.te, W.half_life, W.q, W.z)
    out = torch.zeros((W.J, ldy), dtype=torch.float32)
    out[:, :L] = torch.from_numpy(y)
    return out.cuda()


class BatchPipeline:
    """Many scans in one pass: per-scan prior draws and simulations, one
    batched discrepancy + top-k call for all scans (persistent fused kernel),
    then per-scan model selection and summaries.  `capture()` records the
    whole step into a CUDA graph; `replay()` runs it."""

    def __init__(self, scans: list, precision: int = _lib.ABC_BF16_RESCORE, tuning: dict | None = None):
        self.scans = scans
        self.precision = precision
        self.runs = [AbcPipeline(W, precision, own_workspace=False) for W in scans]   # one batch workspace
        self.ys = [None] * len(scans)
        self.tuning = tuning
        self.graph = None
        self._scan_structs = None
        self.ws = None

    def set_inputs(self, ys):
        self.ys = list(ys)
        self._build_structs()

    def _build_structs(self):
        S_ = _lib.Scan * len(self.scans)
        arr = S_()
        self._w = []
        for i, (r, y) in enumerate(zip(self.runs, self.ys)):
            w = np.ascontiguousarray(r.weights, np.float32)
            self._w.append(w)
            arr[i] = _lib.Scan(y.data_ptr(), r.J, y.shape[1], r.x.data_ptr(), r.N, r.x.shape[1], r.L,
                               w.ctypes.data, r.k, r.idx.data_ptr(), r.dist.data_ptr())
        self._scan_structs = arr
        n = _lib.lib().abc_batch_workspace_size(arr, len(self.scans), self.precision)
        if n == 0:
            raise ValueError("abc_batch_workspace_size: unsupported batch")
        if self.ws is None or self.ws.numel() < n:
            self.ws = torch.empty(n, dtype=torch.uint8, device="cuda")

    def _tuning_ptr(self):
        if self.tuning is None:
            return None
        t = self.tuning
        self._t = _lib.Tuning(t["bn"], t["ctas_per_sm"], t["pilot_stride"], t["pilot_factor"])
        return ctypes.byref(self._t)

    def topk(self, stream=None):
        s = torch.cuda.current_stream() if stream is None else stream
        _lib.check(_lib.lib().abc_batch_discrepancy_topk(self._scan_structs, len(self.scans), self.precision,
                                                         self._tuning_ptr(), ctypes.c_void_p(self.ws.data_ptr()),
                                                         self.ws.numel(), ctypes.c_void_p(s.cuda_stream)))

    def step(self, stream=None):
        for r in self.runs:
            r.simulate_draws(stream)
        self.topk(stream)
        for r in self.runs:
            api.model_select(r.idx, r.offsets, r.prob, r.pref, stream=stream)
            pref = r.pref if len(r.W.models) > 1 else None
            api.summarize(r.theta, r.offsets, r.nparams, r.has_ki, [0, 1, 2], r.idx, pref, out=r.summ,
                          stream=stream)

    def capture(self):
        """Record one step into a CUDA graph (after one eager warm-up step)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()

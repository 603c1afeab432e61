"""One pass of the voxelwise ABC hot path on the GPU (Algorithm 1).

    run = AbcPipeline(workload, precision)        # allocates device buffers once
    out = run.step(y_dev)                         # prior -> simulate -> top-k -> select -> summarise

Every stage is a call into the CUDA library; this module only allocates
device memory and sequences the calls on one stream.
"""
from __future__ import annotations

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
    def __init__(self, W: S.Workload, precision: int | None = None, ldtheta: int = 8):
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
        self.ws = api.alloc_workspace(self.J, self.N, self.L, self.k, self.precision)
        self.idx = torch.empty((self.J, self.k), dtype=torch.int32, device=dev)
        self.dist = torch.empty((self.J, self.k), dtype=torch.float32, device=dev)
        M = len(W.models)
        self.prob = torch.empty((self.J, M), dtype=torch.float32, device=dev)
        self.pref = torch.empty(self.J, dtype=torch.int8, device=dev)
        nc = max(self.nparams) + 1
        self.summ = [torch.empty((self.J, nc), dtype=torch.float32, device=dev) for _ in range(4)]
        self.weights = W.weights.astype(np.float32)

    def simulate_draws(self, stream=None):
        """Algorithm 1, steps 1-3: prior draws and their TACs for every model."""
        W = self.W
        for m, model in enumerate(W.models):
            a, b = self.offsets[m], self.offsets[m + 1]
            lo, hi = W.priors(model)
            api.sample_prior(W.prior_seed, model, lo, hi, b - a, 0, out=self.theta[a:b], stream=stream)
            api.simulate(model, W.ts, W.te, W.inp, self.theta[a:b], out=self.x[a:b], stream=stream)

    def select(self, y, stream=None):
        """Algorithm 1, steps 4-5 plus model probabilities and summaries."""
        api.discrepancy_topk(y, self.x, self.L, self.weights, self.k, self.precision, self.ws, self.idx, self.dist,
                             stream=stream)
        api.model_select(self.idx, self.offsets, self.prob, self.pref, stream=stream)
        pref = self.pref if len(self.W.models) > 1 else None
        api.summarize(self.theta, self.offsets, self.nparams, self.has_ki, [0, 1, 2], self.idx, pref, out=self.summ,
                      stream=stream)

    def step(self, y, stream=None) -> StepOutput:
        self.simulate_draws(stream)
        self.select(y, stream)
        return StepOutput(self.idx, self.dist, self.prob, self.pref, *self.summ)


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
        xc = api.simulate(model, W.ts, W.te, W.inp, torch.from_numpy(np.ascontiguousarray(th)).cuda(), stream=stream)
        x_clean[rows] = xc[:, :L].cpu().numpy()
    y = S.add_noise(x_clean, W.ts, W.te, W.half_life, W.q, W.z)
    out = torch.zeros((W.J, ldy), dtype=torch.float32)
    out[:, :L] = torch.from_numpy(y)
    return out.cuda()

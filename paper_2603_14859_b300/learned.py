"""Learned proposal + importance-weighted local ABC for the irreversible 2TCM.

A build extra with no counterpart in the paper.  A network trained on
simulated (TAC, parameter) pairs predicts, per voxel, a truncated Gaussian over
the unit prior box; local ABC then draws M proposals per voxel from it instead
of scanning the global draw set, and weights the k nearest by prior/proposal.
Voxels where the local run looks unreliable (few effective samples, or a
median accepted distance above what the global path reaches) fall back to the
global path of Algorithm 1 (discrepancy + top-k + summaries).

Every step runs in the CUDA library; this module only sequences the calls and
keeps the buffers.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import _lib
from . import api
from . import synth as S

P = 4            # K1, k2, k3, Vb
NCOL = P + 1     # ... and K_i


@dataclasses.dataclass
class TrainLog:
    steps: int
    pairs: int
    seconds: float
    losses: list


class LearnedLocalAbc:
    """Network + G table + local ABC for one scan (frames, plasma input, noise model)."""

    def __init__(self, ts, te, inp: S.PolyExp, half_life: float, lo=None, hi=None, hidden: int = 256,
                 seed: int = 5005, table_size: int = 512, q_lo: float = 0.10, q_hi: float = 0.10):
        self.ts = np.asarray(ts, np.float64)
        self.te = np.asarray(te, np.float64)
        self.L = len(self.ts)
        self.ldx = ((self.L + 3) // 4) * 4
        self.inp = inp
        self.half_life = half_life
        plo, phi = S.PRIORS[S.TCM2_IRR]
        self.lo = np.asarray(plo if lo is None else lo, np.float64)
        self.hi = np.asarray(phi if hi is None else hi, np.float64)
        self.w = S.frame_weights(self.ts, self.te).astype(np.float32)
        self.D = self.L + 1
        self.H = hidden
        self.O = 2 * P
        self.seed = seed
        self.q_lo, self.q_hi = q_lo, q_hi
        self.params = api.mlp_init(seed, self.D, self.H, self.O)
        self.T = table_size
        self.a_max = float(self.hi[1] + self.hi[2])
        self.table, self.cp_frames = self._build_table()

    # ------------------------------------------------------------------ G table
    def _build_table(self):
        """G(a_i) rows (frame means of e^{-a_i t} (*) C_p) and the frame means of C_p,
        all simulated by the library's 2TCM-irr simulator with special parameter rows."""
        T = self.T
        a = self.a_max * (np.arange(T, dtype=np.float64) / (T - 1)) ** 2
        th = np.zeros((T + 1, 8), np.float32)
        th[:T, 0] = 1.0
        th[:T, 1] = a                       # K1 = 1, k2 = a, k3 = 0, Vb = 0: e^{-a t} (*) C_p
        th[0, 1], th[0, 2] = 0.0, 1.0       # K1 = 1, k2 = 0, k3 = 1: 1 (*) C_p
        th[T] = [1.0, 1.0, 1.0, 1.0, 0, 0, 0, 0]   # Vb = 1: C_p itself
        th_d = torch.from_numpy(th).cuda()
        x = api.simulate(S.TCM2_IRR, self.ts, self.te, self.inp, th_d, ldx=self.L)
        table = api.local_abc_table(x[:T])          # (L, T), frame-major
        cp = x[T].contiguous()
        # the grid must be the fp32 one the kernel assumes: a_i rounded to fp32 exactly as above
        return table, cp

    # ------------------------------------------------------------------ training
    def train(self, n_pairs: int, batch: int = 8192, lr: float = 2e-3, lr_final: float = 1e-4,
              warmup: int = 100, log_every: int = 100, seed: int = 7007) -> TrainLog:
        """Adam on the mean truncated-normal NLL over freshly simulated noisy pairs
        (prior draws -> TACs -> Sec. III-A noise), n_pairs in total."""
        steps = max(1, n_pairs // batch)
        B = batch
        dev = dict(device="cuda", dtype=torch.float32)
        theta = torch.empty((B, 8), **dev)
        x = torch.empty((B, self.ldx), **dev)
        y = torch.empty((B, self.ldx), **dev)
        X = torch.empty((B, self.D), **dev)
        Tt = torch.empty((B, P), **dev)
        grad = torch.empty_like(self.params)
        m = torch.zeros_like(self.params)
        v = torch.zeros_like(self.params)
        loss = torch.empty(1, **dev)
        work = torch.empty(api.mlp_workspace_size(self.D, self.H, self.O, B), dtype=torch.uint8, device="cuda")
        losses = []
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for s in range(steps):
            first = s * B
            api.sample_prior(seed, S.TCM2_IRR, self.lo, self.hi, B, first_index=first, out=theta)
            api.simulate(S.TCM2_IRR, self.ts, self.te, self.inp, theta, out=x)
            api.add_noise(x, self.ts, self.te, self.half_life, self.q_lo, self.q_hi, seed + 1, first_index=first,
                          out=y)
            api.mlp_features(y, self.L, self.w, out=X)
            api.unit_box(theta, B, P, self.lo, self.hi, out=Tt)
            api.mlp_loss_grad(self.params, self.D, self.H, P, X, Tt, grad=grad, loss=loss, work=work)
            frac = s / max(1, steps - 1)
            lr_s = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * frac))
            if s < warmup:
                lr_s *= (s + 1) / warmup
            api.adam_update(self.params, grad, m, v, lr_s, s + 1)
            if log_every and (s % log_every == 0 or s == steps - 1):
                losses.append((s, float(loss.item())))
        t1.record()
        torch.cuda.synchronize()
        return TrainLog(steps, steps * B, t0.elapsed_time(t1) / 1e3, losses)

    # ------------------------------------------------------------------ inference
    def propose(self, y, chunk: int = 262144, out=None):
        """Network outputs (J x 8: mu, log sigma per parameter) for the voxel TACs y."""
        J = y.shape[0]
        if out is None:
            out = torch.empty((J, self.O), device="cuda", dtype=torch.float32)
        c = min(chunk, max(J, 1))
        X = torch.empty((c, self.D), device="cuda", dtype=torch.float32)
        work = torch.empty(api.mlp_workspace_size(self.D, self.H, self.O, c), dtype=torch.uint8, device="cuda")
        for j0 in range(0, J, c):
            n = min(c, J - j0)
            api.mlp_features(y[j0:j0 + n], self.L, self.w, out=X[:n])
            api.mlp_forward(self.params, self.D, self.H, self.O, X[:n], out=out[j0:j0 + n], work=work)
        return out

    def local(self, y, prop, M: int = 10_000, k: int = 200, seed: int = 9009, sigma_scale: float = 1.0,
              dump: bool = False, out=None):
        return api.local_abc(y, self.L, self.w, prop, self.table, self.a_max, self.cp_frames, self.lo, self.hi, M, k,
                             seed, sigma_scale=sigma_scale, dump=dump, out=out)

    @staticmethod
    def uniform_proposal(J):
        """Proposal parameters that make q nearly flat on the box (mu = 0.5, sigma = e^2):
        local ABC with them is plain rejection ABC on M prior-like draws."""
        p = torch.empty((J, 2 * P), device="cuda", dtype=torch.float32)
        p[:, 0::2] = 0.5
        p[:, 1::2] = 2.0
        return p


class GlobalIrr:
    """The global path (Algorithm 1) for the irreversible 2TCM, used for
    calibration and as the fallback of the learned path."""

    def __init__(self, model: LearnedLocalAbc, N: int, k: int, seed: int = 1234,
                 precision: int = _lib.ABC_BF16_RESCORE):
        self.m = model
        self.N, self.k, self.precision = N, k, precision
        self.theta = api.sample_prior(seed, S.TCM2_IRR, model.lo, model.hi, N)
        self.x = api.simulate(S.TCM2_IRR, model.ts, model.te, model.inp, self.theta)
        self.offsets = [0, N]
        self.ws = None

    def reserve(self, J):
        """Keep a workspace for up to J voxels (reused across calls)."""
        need = api.workspace_size(J, self.N, self.m.L, self.k, self.precision)
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device="cuda")

    def run(self, y):
        self.reserve(y.shape[0])
        idx, dist = api.discrepancy_topk(y, self.x, self.m.L, self.m.w, self.k, self.precision, workspace=self.ws)
        mean, sd, lo, hi = api.summarize(self.theta, self.offsets, [P], [1], [0, 1, 2], idx)
        return dict(idx=idx, dist=dist, mean=mean, sd=sd, lo=lo, hi=hi)

    def calibrate(self, y, quantile: float = 0.99) -> float:
        """Relative median accepted distance (d_med / sum w y^2) the global path
        reaches on these voxels, at the given quantile (computed by the library)."""
        r = self.run(y)
        return api.median_rel_quantile(r["dist"], self.k, y, self.m.L, self.m.w, quantile)


def fallback_to_global(out, y, k: int, global_path: GlobalIrr, rel_max: float | None):
    """Voxels whose local run is unreliable (the library's predicate: ESS below k/4, or a
    median accepted distance above rel_max sum w y^2) take the global path's summaries, in
    place in out.  Returns the fallback voxels (device int32, ascending) and their number."""
    rows, count = api.fallback_rows(out["ess"], out["dmed"], out["ynorm"], k, rel_max)
    n = int(count.item())
    if n > 0:
        g = global_path.run(api.gather_rows(y, rows, count, n))
        for key in ("mean", "sd", "lo", "hi"):
            api.scatter_rows(g[key], rows, count, out[key])
    return rows[:n], n


def run_learned(model: LearnedLocalAbc, y, M: int, k: int, global_path: GlobalIrr | None, rel_max: float | None,
                seed: int = 9009, sigma_scale: float = 1.0):
    """Learned proposal -> local ABC -> fallback of unreliable voxels to the global path.
    Returns (outputs dict, fallback voxel indices)."""
    prop = model.propose(y)
    out = model.local(y, prop, M=M, k=k, seed=seed, sigma_scale=sigma_scale)
    fb = torch.zeros(0, dtype=torch.int32, device="cuda")
    if global_path is not None:
        fb, _ = fallback_to_global(out, y, k, global_path, rel_max)
    out["prop"] = prop
    return out, fb

"""Seeded synthetic inputs for voxelwise ABC on dynamic PET.

This module generates workload data only: frame schedules, plasma-input
parameters, reference-tissue input, ground-truth kinetic parameters, noise
levels and standard-normal noise draws, plus the noise model that turns a
clean TAC into a measured one.  It holds none of the inference arithmetic
(prior sampling, TAC simulation, distances, top-k, summaries): those live in
the CUDA library and, independently, in the FP64 test oracle.  Both sides take
their inputs from here.

Every generator takes an explicit seed and uses numpy's Philox bit generator,
so a workload is reproducible from its name and seed.

Units: time in minutes, rate constants in 1/min.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Model identifiers (same numbering as the C ABI).
TCM2_IRR = 0
TCM2_REV = 1
MRTM = 2
LPNTPET = 3
MODEL_NAMES = {TCM2_IRR: "2TCM-irr", TCM2_REV: "2TCM-rev", MRTM: "MRTM", LPNTPET: "lp-ntPET"}

# Parameter order per model.  2TCM: Sec. III-A ranges (K1, k2, k3, [k4,] Vb).
# MRTM / lp-ntPET: (R1, k2, BP_ND[, gamma, t_D, t_P - t_D, alpha]); the
# simulator derives k2a = k2 / (1 + BP_ND) (Sec. II-A, Eq. 3).
PARAM_NAMES = {
    TCM2_IRR: ["K1", "k2", "k3", "Vb"],
    TCM2_REV: ["K1", "k2", "k3", "k4", "Vb"],
    MRTM: ["R1", "k2", "BPnd"],
    LPNTPET: ["R1", "k2", "BPnd", "gamma", "tD", "tPmD", "alpha"],
}

# Uniform prior boxes.  2TCM: Sec. III-A / Eq. prior2.  Reference-tissue models:
# the paper defers to the literature; these boxes are this project's reading.
PRIORS = {
    TCM2_IRR: ([0.001, 0.001, 0.001, 0.03], [1.0, 2.0, 0.5, 0.20]),
    TCM2_REV: ([0.001, 0.001, 0.001, 0.0, 0.03], [1.0, 2.0, 0.5, 0.10, 0.20]),
    MRTM: ([0.6, 0.1, 0.0], [1.6, 0.6, 4.0]),
    LPNTPET: ([0.6, 0.1, 0.0, 0.0, 20.0, 1.0, 0.25], [1.6, 0.6, 4.0, 0.3, 45.0, 15.0, 4.0]),
}

# Feng plasma-input parameter ranges (Sec. III-A).
FENG_LO = dict(b1=4e4, b2=1e4, b3=8e3, k1=1.0, k2=0.03, k3=0.01)
FENG_HI = dict(b1=4.7e5, b2=2e5, b3=3e4, k1=1e3, k2=3.60, k3=0.035)

HALF_LIFE_F18 = 109.8   # min (Sec. III-A)
HALF_LIFE_C11 = 20.4    # min (physical constant; the paper names the tracer only)

# 1-tissue reference region used to build C_r for the reference-tissue models.
REF_K1 = 0.1
REF_K2 = 0.35


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


# --------------------------------------------------------------------------- frames
def frames_from_blocks(blocks_s):
    """Contiguous frame schedule from (count, seconds) blocks, in minutes."""
    edges = [0.0]
    for count, sec in blocks_s:
        for _ in range(count):
            edges.append(edges[-1] + sec / 60.0)
    e = np.asarray(edges, dtype=np.float64)
    return e[:-1].copy(), e[1:].copy()


def frames_brain_fdg22():
    """22 frames: 6x10 s, 4x30 s, 4x60 s, 4x300 s, 4x300 s (47 min as listed)."""
    return frames_from_blocks([(6, 10), (4, 30), (4, 60), (4, 300), (4, 300)])


def frames_raclopride60():
    """60 one-minute frames."""
    return frames_from_blocks([(60, 60)])


def frames_totalbody29():
    """29 frames over 50 min: 6x10 s, 6x30 s, 6x60 s, 5x120 s, 6x300 s."""
    return frames_from_blocks([(6, 10), (6, 30), (6, 60), (5, 120), (6, 300)])


def frames_uneven(F: int):
    """F frames: 6x10 s, 4x30 s, 4x60 s, then F-14 equal frames up to 60 min."""
    assert F >= 15
    ts, te = frames_from_blocks([(6, 10), (4, 30), (4, 60)])
    rest = np.linspace(te[-1], 60.0, F - 14 + 1)
    return np.concatenate([ts, rest[:-1]]), np.concatenate([te, rest[1:]])


def frame_weights(ts, te):
    """Frame-duration weights w_l = dt_l / sum(dt)."""
    dt = np.asarray(te) - np.asarray(ts)
    return dt / dt.sum()


# --------------------------------------------------------------------------- inputs
@dataclasses.dataclass
class PolyExp:
    """Input function sum_i (a0_i + a1_i t + a2_i t^2) exp(-c_i t)."""
    c: np.ndarray
    a0: np.ndarray
    a1: np.ndarray
    a2: np.ndarray

    @property
    def n_terms(self):
        return len(self.c)


def draw_feng(seed: int, avoid=None, min_gap=0.05):
    """One Feng parameter set (beta1..3, kappa1..3) uniform over Sec. III-A ranges.

    `avoid` lists rates the kappas must stay `min_gap` away from (used when the
    input is later convolved with a fixed reference-tissue rate, so that the
    reference TAC's own partial fractions stay well conditioned)."""
    rng = _rng(seed, 11)
    while True:
        b = [rng.uniform(FENG_LO[k], FENG_HI[k]) for k in ("b1", "b2", "b3")]
        kap = [rng.uniform(FENG_LO[k], FENG_HI[k]) for k in ("k1", "k2", "k3")]
        if avoid is None or all(abs(kk - a) > min_gap for kk in kap for a in avoid):
            return np.array(b), np.array(kap)


def feng_polyexp(beta, kappa) -> PolyExp:
    """Feng input (Sec. III-A) as three poly-exponential terms."""
    b1, b2, b3 = beta
    k1, k2, k3 = kappa
    return PolyExp(c=np.array([k1, k2, k3], float), a0=np.array([-b2 - b3, b2, b3], float),
                   a1=np.array([b1, 0.0, 0.0]), a2=np.zeros(3))


def reference_tissue_polyexp(cp: PolyExp, K1=REF_K1, k2=REF_K2) -> PolyExp:
    """C_r = K1' * (C_p conv exp(-k2' t)) written out as a poly-exponential.

    Workload construction for the reference-region TAC of the reference-tissue
    models (a 1-tissue region).  Supports input terms up to t^1."""
    assert np.all(cp.a2 == 0)
    c, a0, a1 = [], [], []
    coef_k = 0.0
    for ci, p0, p1 in zip(cp.c, cp.a0, cp.a1):
        d = ci - k2
        # conv(exp(-k2 t), p0 exp(-c t)) = p0 (exp(-k2 t) - exp(-c t)) / d
        coef_k += p0 / d
        t0 = -p0 / d
        # conv(exp(-k2 t), p1 t exp(-c t)) = p1 [exp(-k2 t) - exp(-c t) - d t exp(-c t)] / d^2
        coef_k += p1 / d**2
        t0 += -p1 / d**2
        t1 = -p1 / d
        c.append(ci)
        a0.append(K1 * t0)
        a1.append(K1 * t1)
    c.append(k2)
    a0.append(K1 * coef_k)
    a1.append(0.0)
    return PolyExp(np.array(c), np.array(a0), np.array(a1), np.zeros(len(c)))


# --------------------------------------------------------------------------- truth
def uniform_truth(seed: int, model: int, J: int, lo=None, hi=None) -> np.ndarray:
    """Ground-truth parameters uniform over a box (float32, J x P)."""
    plo, phi = PRIORS[model]
    lo = np.asarray(plo if lo is None else lo, float)
    hi = np.asarray(phi if hi is None else hi, float)
    rng = _rng(seed, 21 + model)
    return (lo + (hi - lo) * rng.random((J, len(lo)))).astype(np.float32)


def cluster_truth(seed: int, model: int, J: int, n_clusters=8, sigma_log=0.25) -> np.ndarray:
    """Organ-like ground truth: lognormal clusters inside the prior box (J x P)."""
    plo, phi = PRIORS[model]
    lo, hi = np.asarray(plo, float), np.asarray(phi, float)
    rng = _rng(seed, 31 + model)
    P = len(lo)
    # cluster log-medians spread across the interior of the box
    lo_pos = np.maximum(lo, 1e-3)
    u = rng.uniform(0.15, 0.85, (n_clusters, P))
    med = np.exp(np.log(lo_pos) + u * (np.log(hi) - np.log(lo_pos)))
    lab = rng.integers(0, n_clusters, J)
    th = med[lab] * np.exp(sigma_log * rng.standard_normal((J, P)))
    th = np.clip(th, lo, hi)
    return th.astype(np.float32), lab


def noise_levels(seed: int, J: int, q_lo: float, q_hi: float) -> np.ndarray:
    if q_lo == q_hi:
        return np.full(J, q_lo, np.float64)
    return _rng(seed, 41).uniform(q_lo, q_hi, J)


def standard_normals(seed: int, J: int, L: int) -> np.ndarray:
    return _rng(seed, 51).standard_normal((J, L))


def add_noise(x_clean: np.ndarray, ts, te, half_life: float, q: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Gaussian decay-weighted noise (Sec. III-A): y = x + l_v sigma z, with
    sigma_l = sqrt(x_l exp(lambda t_mid,l) / dt_l) and the per-voxel level l_v
    chosen so that ||l_v sigma|| = q ||x||.  Returns float32."""
    ts, te = np.asarray(ts), np.asarray(te)
    lam = math.log(2.0) / half_life
    dt = te - ts
    tm = 0.5 * (ts + te)
    x = np.asarray(x_clean, np.float64)
    sig = np.sqrt(np.maximum(x, 0.0) * np.exp(lam * tm) / dt)
    nrm_s = np.sqrt((sig**2).sum(1))
    nrm_x = np.sqrt((x**2).sum(1))
    lv = np.where(nrm_s > 0, q * nrm_x / np.where(nrm_s > 0, nrm_s, 1.0), 0.0)
    return (x + lv[:, None] * sig * z).astype(np.float32)


def poisson_scale(x_clean: np.ndarray, q: float) -> float:
    """Counting-noise constant l2 at which the median voxel's Poisson noise has
    relative size q: E||y - x||^2 = sum_l x_l / l2 = q^2 ||x||^2 (the paper estimates
    its l2 from scanner data, which this build does not have)."""
    x = np.maximum(np.asarray(x_clean, np.float64), 0.0)
    r = x.sum(1) / np.maximum((x * x).sum(1), 1e-300)
    return float(np.median(r) / (q * q))


def add_noise_poisson(x_clean: np.ndarray, l2: float, seed: int) -> np.ndarray:
    """Poisson counting noise of the lp-ntPET simulation study (Sec. IV-A):
    y_l = Pois(l2 x_l) / l2, mean x_l and variance x_l / l2.  Returns float32."""
    x = np.maximum(np.asarray(x_clean, np.float64), 0.0)
    return (_rng(seed, 71).poisson(l2 * x) / l2).astype(np.float32)


def mask_indices(shape, J: int) -> np.ndarray:
    """Linear indices of the J voxels closest to the centre of an ellipsoid
    inscribed in `shape` (a compact voxel list for a masked volume)."""
    axes = [np.linspace(-1.0, 1.0, s) for s in shape]
    g = np.meshgrid(*axes, indexing="ij")
    r2 = sum(a * a for a in g).ravel()
    idx = np.argpartition(r2, J - 1)[:J]
    return np.sort(idx).astype(np.int64)


# --------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class Workload:
    name: str
    ts: np.ndarray
    te: np.ndarray
    models: list            # candidate model ids, in index order of the draw segments
    n_per_model: list       # draws per model
    k: int
    inp: PolyExp            # C_p (2TCM) or C_r (reference-tissue models)
    half_life: float
    truth_model: np.ndarray  # (J,) int
    truth: list             # per model: (J_m x P_m) float32 truth rows for voxels of that model
    truth_rows: list        # per model: voxel indices owning those rows
    q: np.ndarray           # (J,) noise level
    z: np.ndarray           # (J, L) standard normals
    prior_seed: int
    precision: str = "fp32"
    model_inp: dict | None = None  # per-model input when the models need different ones
    noise: str = "gaussian"        # "gaussian": add_noise with levels q; "poisson": add_noise_poisson
    noise_q: float = 0.0           # poisson: relative noise size of the median voxel (sets l2)
    noise_seed: int = 0

    def input_for(self, model):
        if self.model_inp and model in self.model_inp:
            return self.model_inp[model]
        return self.inp

    @property
    def L(self):
        return len(self.ts)

    @property
    def J(self):
        return len(self.q)

    @property
    def N(self):
        return int(sum(self.n_per_model))

    @property
    def weights(self):
        return frame_weights(self.ts, self.te)

    def model_offsets(self):
        off = [0]
        for n in self.n_per_model:
            off.append(off[-1] + int(n))
        return off

    def priors(self, model):
        lo, hi = PRIORS[model]
        return np.asarray(lo, float), np.asarray(hi, float)


def workload(name: str, seed: int | None = None, J: int | None = None, N_per_model: int | None = None,
             noise: str = "gaussian", level: str = "high") -> Workload:
    """Named synthetic workload.  `J` and `N_per_model` shrink it for tests; `noise`
    and `level` select the noise model of the lp-ntPET detection study."""
    if name == "brain_fdg_2tcm":            # plain ABC, 2TCM-irr, 22 frames
        seed = 1001 if seed is None else seed
        J = 2048 if J is None else J
        n = 50_000 if N_per_model is None else N_per_model
        ts, te = frames_brain_fdg22()
        beta, kap = draw_feng(seed)
        truth = uniform_truth(seed, TCM2_IRR, J)
        return Workload(name, ts, te, [TCM2_IRR], [n], 100, feng_polyexp(beta, kap), HALF_LIFE_F18,
                        np.zeros(J, np.int32), [truth], [np.arange(J)], noise_levels(seed, J, 0.10, 0.10),
                        standard_normals(seed, J, len(ts)), seed + 7, "fp32")
    if name == "raclopride_lpntpet":        # MRTM vs lp-ntPET model selection, 60 frames
        seed = 1002 if seed is None else seed
        J = 250_000 if J is None else J
        n = 1_000_000 if N_per_model is None else N_per_model
        ts, te = frames_raclopride60()
        beta, kap = draw_feng(seed, avoid=[REF_K2])
        cr = reference_tissue_polyexp(feng_polyexp(beta, kap))
        rng = _rng(seed, 61)
        act = rng.random(J) < 0.05
        tm = np.where(act, LPNTPET, MRTM).astype(np.int32)
        rows_a = np.nonzero(act)[0]
        rows_m = np.nonzero(~act)[0]
        lo, hi = PRIORS[LPNTPET]
        lo = list(lo); lo[3] = 0.05                  # activated voxels carry a visible gamma
        th_a = uniform_truth(seed, LPNTPET, len(rows_a), lo, hi)
        th_m = uniform_truth(seed, MRTM, len(rows_m))
        return Workload(name, ts, te, [MRTM, LPNTPET], [n, n], 500, cr, HALF_LIFE_C11, tm,
                        [th_m, th_a], [rows_m, rows_a], noise_levels(seed, J, 0.05, 0.20),
                        standard_normals(seed, J, len(ts)), seed + 7, "bf16r")
    if name == "raclopride_e2":             # lp-ntPET detection study: 61 one-minute frames, half activated
        seed = 1006 if seed is None else seed
        J = 4000 if J is None else J
        n = 1_000_000 if N_per_model is None else N_per_model
        ts, te = frames_from_blocks([(61, 60)])
        beta, kap = draw_feng(seed, avoid=[REF_K2])
        cr = reference_tissue_polyexp(feng_polyexp(beta, kap))
        act = np.zeros(J, bool)
        act[_rng(seed, 61).permutation(J)[: J // 2]] = True
        tm = np.where(act, LPNTPET, MRTM).astype(np.int32)
        rows_a, rows_m = np.nonzero(act)[0], np.nonzero(~act)[0]
        lo, hi = PRIORS[LPNTPET]
        lo = list(lo); lo[3] = 0.05
        th_a = uniform_truth(seed, LPNTPET, len(rows_a), lo, hi)
        th_m = uniform_truth(seed, MRTM, len(rows_m))
        q = {"low": 0.03, "high": 0.10}[level]
        if noise not in ("gaussian", "poisson"):
            raise KeyError(noise)
        return Workload(name, ts, te, [MRTM, LPNTPET], [n, n], 500, cr, HALF_LIFE_C11, tm,
                        [th_m, th_a], [rows_m, rows_a], noise_levels(seed, J, q, q),
                        standard_normals(seed, J, len(ts)), seed + 7, "bf16r", noise=noise, noise_q=q,
                        noise_seed=seed + 11)
    if name == "totalbody_fdg":             # 2TCM irr vs rev, 29 frames, lognormal clusters
        seed = 1003 if seed is None else seed
        J = 4_000_000 if J is None else J
        n = 1_000_000 if N_per_model is None else N_per_model
        ts, te = frames_totalbody29()
        beta, kap = draw_feng(seed)
        rng = _rng(seed, 62)
        rev = rng.random(J) < 0.30
        tm = np.where(rev, TCM2_REV, TCM2_IRR).astype(np.int32)
        rows_i, rows_r = np.nonzero(~rev)[0], np.nonzero(rev)[0]
        th_i, _ = cluster_truth(seed, TCM2_IRR, len(rows_i))
        th_r, _ = cluster_truth(seed, TCM2_REV, len(rows_r))
        th_r[:, 3] = _rng(seed, 63).uniform(0.005, 0.1, len(rows_r)).astype(np.float32)
        return Workload(name, ts, te, [TCM2_IRR, TCM2_REV], [n, n], 200, feng_polyexp(beta, kap),
                        HALF_LIFE_F18, tm, [th_i, th_r], [rows_i, rows_r], noise_levels(seed, J, 0.10, 0.10),
                        standard_normals(seed, J, len(ts)), seed + 7, "bf16r")
    raise KeyError(name)


def scan_plan(seed: int = 1004, n_scans: int = 64, voxel_scale: float = 1.0, draw_scale: float = 1.0):
    """Batched uneven workload: per scan (voxels, frames, candidate models, draws)."""
    rng = _rng(seed, 71)
    plan = []
    for s in range(n_scans):
        J = int(round(math.exp(rng.uniform(math.log(1_000), math.log(500_000))) * voxel_scale))
        F = int(rng.integers(22, 61))
        nm = int(rng.integers(1, 4))
        models = sorted(rng.choice([TCM2_IRR, TCM2_REV, MRTM], nm, replace=False).tolist())
        n = [int(round(rng.uniform(200_000, 1_000_000) * draw_scale)) for _ in models]
        plan.append(dict(scan=s, J=max(J, 1), F=F, models=models, n_per_model=n, seed=seed * 1000 + s))
    return plan


def scan_workload(item: dict, k: int = 100) -> Workload:
    """One scan of the batched uneven workload (an entry of `scan_plan`).

    Frames: `frames_uneven(F)`.  Inputs: a seeded Feng C_p for the 2TCM
    models and the 1-tissue reference C_r built from it for MRTM.  Truth: each
    voxel follows one of the scan's candidate models (uniformly), parameters
    uniform over that model's prior box; noise level q = 0.10."""
    seed = item["seed"]
    J = item["J"]
    ts, te = frames_uneven(item["F"])
    beta, kap = draw_feng(seed, avoid=[REF_K2])
    cp = feng_polyexp(beta, kap)
    cr = reference_tissue_polyexp(cp)
    models = list(item["models"])
    inputs = {m: (cr if m == MRTM else cp) for m in models}
    rng = _rng(seed, 81)
    pick = rng.integers(0, len(models), J)
    tm = np.asarray(models)[pick].astype(np.int32)
    truth, rows = [], []
    for m in models:
        r = np.nonzero(tm == m)[0]
        rows.append(r)
        truth.append(uniform_truth(seed, m, len(r)))
    n = [int(v) for v in item["n_per_model"]]
    kk = min(k, sum(n))
    half = HALF_LIFE_C11 if models == [MRTM] else HALF_LIFE_F18
    return Workload(f"scan{item['scan']}", ts, te, models, n, kk, cp, half, tm, truth, rows,
                    noise_levels(seed, J, 0.10, 0.10), standard_normals(seed, J, len(ts)), seed + 7, "bf16r",
                    model_inp=inputs)

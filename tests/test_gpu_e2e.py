"""End-to-end parity: prior draws, simulation, discrepancy, top-k, model selection and
summaries (Alg. 1 steps 1-5; Sec. II-D point estimates and 95 % credible intervals;
Sec. III-B K_i and model probabilities).

The oracle draws the same Philox prior stream, simulates every draw with its own FP64
integrators, ranks the draws by the directly computed distance and summarises; the GPU
pipeline does all of it with its own kernels.  The two simulators agree to 2e-6 of each
TAC's peak for the closed forms and 1e-4 for lp-ntPET (the simulator parity tests), so
an accepted set may differ from the oracle's only by draws whose oracle distance lies
within the band that this difference allows around the k-th distance: with
Delta_n = eps_model * peak_n >= the weighted norm of the TAC difference of draw n,
|sqrt(d_n) - sqrt(d_(k))| <= 2 (Delta_n + max over the accepted draws of Delta) plus the
fp32 near-tie band.  Where the sets are equal, model probabilities and summaries agree
within 1e-5 relative.  Workloads: the brain FDG 2TCM-irr case in full (2,048 voxels x
50,000 draws) and 512-voxel x 100,000-draw slices of the brain lp-ntPET / MRTM and
total-body FDG workloads, in every precision form."""
import numpy as np
import pytest
import torch

from paper_2603_14859_b300 import synth as S

pytestmark = pytest.mark.gpu

SIM_EPS = {S.TCM2_IRR: 2e-6, S.TCM2_REV: 2e-6, S.MRTM: 2e-6, S.LPNTPET: 1e-4}
CASES = [("brain_fdg_2tcm", None, None), ("raclopride_lpntpet", 512, 50_000), ("totalbody_fdg", 512, 50_000)]
_ORACLE = {}


def _oracle_side(orc, name, J, n):
    """Everything the oracle computes for a case, from the workload's seeds alone."""
    key = (name, J, n)
    if key in _ORACLE:
        return _ORACLE[key]
    W = S.workload(name, J=J, N_per_model=n)
    L = W.L
    off = W.model_offsets()
    thetas, xs, eps = [], [], []
    for m, model in enumerate(W.models):
        lo, hi = W.priors(model)
        th = orc.sample_prior(W.prior_seed, model, lo, hi, off[m + 1] - off[m], ldtheta=8)
        x = orc.simulate(model, W.ts, W.te, W.input_for(model), th)
        thetas.append(th)
        xs.append(x)
        eps.append(SIM_EPS[model] * np.abs(x).max(1))
    theta, X, delta = np.concatenate(thetas), np.concatenate(xs), np.concatenate(eps)
    xc = np.zeros((W.J, L))
    for th, rows in zip(W.truth, W.truth_rows):
        if len(rows):
            xc[rows] = orc.simulate(int(W.truth_model[rows[0]]), W.ts, W.te, W.input_for(int(W.truth_model[rows[0]])), th)
    y = S.add_noise(xc, W.ts, W.te, W.half_life, W.q, W.z)
    w = W.weights
    idx, dist = orc.topk(y, X, w, W.k)
    prob, pref = orc.model_select(idx, off)
    nparams = [len(S.PARAM_NAMES[m]) for m in W.models]
    has_ki = [1 if m in (S.TCM2_IRR, S.TCM2_REV) else 0 for m in W.models]
    summ = orc.summarize(theta, off, nparams, has_ki, [0, 1, 2], idx, pref if len(W.models) > 1 else None)
    out = dict(W=W, theta=theta, X=X, delta=delta, y=y, idx=idx, dist=dist, prob=prob, pref=pref, summ=summ)
    _ORACLE[key] = out
    return out


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name,J,n", CASES)
def test_end_to_end_against_oracle(orc, name, J, n, prec):
    from paper_2603_14859_b300 import api, pipeline
    o = _oracle_side(orc, name, J, n)
    W = o["W"]
    L, k = W.L, W.k
    run = pipeline.AbcPipeline(W, prec)
    ld = run.ldx
    yp = np.zeros((W.J, ld), np.float32)
    yp[:, :L] = o["y"]
    out = run.step(torch.from_numpy(yp).cuda())
    torch.cuda.synchronize()
    assert api.topk_status(run.ws)[0] == 0
    # prior draws: the same Philox stream, bit for bit
    assert np.array_equal(run.theta.cpu().numpy(), o["theta"])
    gi = out.idx.cpu().numpy()
    oi, od, X, delta = o["idx"], o["dist"], o["X"], o["delta"]
    y32 = o["y"].astype(np.float32)
    same = np.ones(W.J, bool)
    for j in range(W.J):
        g, s_ = set(gi[j].tolist()), set(oi[j].tolist())
        if g == s_:
            continue
        same[j] = False
        diff = np.array(sorted(g ^ s_))
        assert (diff >= 0).all()
        dd = orc.pair_dist(y32, X, W.weights, np.full(len(diff), j), diff)
        sk = np.sqrt(od[j, -1])
        band = 2 * (delta[diff] + delta[oi[j]].max()) + 16 * L * 2.0**-24 * sk
        bad = diff[np.abs(np.sqrt(dd) - sk) > band]
        assert len(bad) == 0, f"voxel {j}: draws {bad[:5]} differ outside the simulator band"
    assert same.mean() > 0.5
    # model probabilities and summaries where the accepted sets agree
    prob_g, pref_g = out.prob.cpu().numpy(), out.pref.cpu().numpy()
    assert np.array_equal(pref_g[same], o["pref"][same])
    assert np.allclose(prob_g[same], o["prob"][same], rtol=0, atol=1e-7)
    table = {}
    for nm, g, ref in zip(("mean", "sd", "lo", "hi"), (out.mean, out.sd, out.lo, out.hi), o["summ"]):
        g = g.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.isnan(g), np.isnan(ref))
        m = ~np.isnan(ref)
        err = np.where(m, np.abs(g - ref) / np.maximum(np.abs(ref), 1e-12), 0.0)
        ok = np.where(m, np.abs(g - ref) <= 1e-5 * np.abs(ref) + 1e-7, True)
        assert ok[same].all(), f"{nm}: summaries differ on voxels with equal accepted sets"
        table[nm] = (float(err[same].max()), float(err.max()))
    perr = float(np.abs(prob_g - o["prob"]).max())
    print(f"\nE2E {name} prec={prec}: voxels {W.J}, equal sets {int(same.sum())}; max rel error "
          f"(equal sets / all voxels): " + ", ".join(f"{k_}={a:.2e}/{b:.2e}" for k_, (a, b) in table.items())
          + f"; model probability max abs error (all voxels) {perr:.3e}")

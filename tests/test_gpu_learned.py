"""Learned proposal + importance-weighted local ABC on the GPU against the FP64
oracle: network forward and gradient, Adam, noise and target kernels, the
truncated-normal sampler, the local ABC stages (distances, accepted set,
weights, summaries), and the gain of the trained network over prior-like
proposals at the same draw budget."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def bf16_round_weights(prm, D, H, O):
    """The weights as the network uses them: W1, W2, W3 rounded to bf16, biases fp32."""
    p = torch.from_numpy(np.asarray(prm, np.float32).copy())
    segs = [(0, H * D), (H * D + H, H * D + H + H * H), (H * D + 2 * H + H * H, H * D + 2 * H + H * H + O * H)]
    for a, b in segs:
        p[a:b] = p[a:b].to(torch.bfloat16).to(torch.float32)
    return p.numpy().astype(np.float64)


@pytest.mark.parametrize("D,H,B", [(30, 80, 300), (23, 64, 64), (30, 256, 2048)])
def test_mlp_forward_and_gradient(orc, D, H, B):
    from paper_2603_14859_b300 import api
    P = 4
    O = 2 * P
    rng = np.random.default_rng(D * 1000 + H + B)
    prm = api.mlp_init(11 + H, D, H, O)
    # non-zero biases so that every bias gradient path is exercised
    nb = prm.cpu().numpy()
    nb[H * D:H * D + H] = rng.normal(0, 0.1, H)
    nb[H * D + H + H * H:H * D + 2 * H + H * H] = rng.normal(0, 0.1, H)
    nb[-O:] = rng.normal(0, 0.3, O)
    prm = torch.from_numpy(nb).cuda()
    X = rng.normal(0, 1, (B, D)).astype(np.float32)
    T = rng.uniform(0, 1, (B, P)).astype(np.float32)
    out = api.mlp_forward(prm, D, H, O, torch.from_numpy(X).cuda()).cpu().numpy()
    pr = bf16_round_weights(nb, D, H, O)
    ref = orc.mlp_forward(pr, D, H, O, X.astype(np.float64))
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 2e-5 * scale + 1e-6
    loss, grad = api.mlp_loss_grad(prm, D, H, P, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    rl, rg = orc.mlp_loss_grad(pr, D, H, P, X.astype(np.float64), T.astype(np.float64))
    assert abs(float(loss.item()) - rl) <= 1e-5 * abs(rl) + 1e-5
    g = grad.cpu().numpy().astype(np.float64)
    # per parameter block: fp32 sums over B rows against the fp64 oracle
    bounds = np.cumsum([0, H * D, H, H * H, H, O * H, O])
    for a, b in zip(bounds[:-1], bounds[1:]):
        err = np.abs(g[a:b] - rg[a:b]).max()
        assert err <= 1e-4 * np.abs(rg[a:b]).max() + 1e-7, (a, b, err)


def test_mlp_gradient_matches_finite_differences_in_loss(orc):
    """The GPU loss moves along the GPU gradient as a first-order model predicts
    (a tiny network, biases only, where bf16 rounding does not apply)."""
    from paper_2603_14859_b300 import api
    D, H, P = 6, 8, 4
    O = 2 * P
    rng = np.random.default_rng(3)
    prm = api.mlp_init(5, D, H, O)
    X = torch.from_numpy(rng.normal(0, 1, (50, D)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.uniform(0.05, 0.95, (50, P)).astype(np.float32)).cuda()
    loss, grad = api.mlp_loss_grad(prm, D, H, P, X, T)
    l0 = float(loss.item())
    g = grad.clone()
    bias_slots = list(range(H * D, H * D + H)) + list(range(len(prm) - O, len(prm)))
    for s in bias_slots[::3]:
        h = 1e-2
        p2 = prm.clone()
        p2[s] += h
        l1 = float(api.mlp_loss_grad(p2, D, H, P, X, T)[0].item())
        p2[s] -= 2 * h
        lm = float(api.mlp_loss_grad(p2, D, H, P, X, T)[0].item())
        fd = (l1 - lm) / (2 * h)
        assert abs(fd - float(g[s])) <= 2e-2 * abs(float(g[s])) + 2e-4, (s, fd, float(g[s]), l0)


def test_adam_step_against_numpy():
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(4)
    n = 1000
    p = rng.normal(0, 1, n).astype(np.float32)
    g = rng.normal(0, 1, n).astype(np.float32)
    m = rng.normal(0, 0.1, n).astype(np.float32)
    v = rng.uniform(0, 0.1, n).astype(np.float32)
    dp, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    api.adam_update(dp, dg, dm, dv, 1e-3, 7, 0.9, 0.999, 1e-8)
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))      # the constants as the kernel receives them
    m2 = b1 * m.astype(np.float64) + (1 - b1) * g
    v2 = b2 * v.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    p2 = p - 1e-3 * (m2 / (1 - b1 ** 7)) / (np.sqrt(v2 / (1 - b2 ** 7)) + 1e-8)
    assert np.allclose(dm.cpu().numpy(), m2, rtol=1e-6, atol=1e-7)
    assert np.allclose(dv.cpu().numpy(), v2, rtol=1e-6, atol=1e-9)
    assert np.allclose(dp.cpu().numpy(), p2, rtol=1e-6, atol=1e-7)


def test_features_targets_and_noise():
    from paper_2603_14859_b300 import api
    from paper_2603_14859_b300 import synth as S
    ts, te = S.frames_totalbody29()
    L = len(ts)
    w = S.frame_weights(ts, te).astype(np.float32)
    rng = np.random.default_rng(5)
    y = rng.uniform(10, 5000, (777, 32)).astype(np.float32)
    f = api.mlp_features(torch.from_numpy(y).cuda(), L, w).cpu().numpy()
    s = np.sqrt((w * y[:, :L].astype(np.float64) ** 2).sum(1))
    assert np.allclose(f[:, :L], y[:, :L] / s[:, None], rtol=1e-5)
    assert np.allclose(f[:, L], np.log(s) / 10, rtol=1e-5, atol=1e-6)
    # unit-box targets
    lo, hi = S.PRIORS[S.TCM2_IRR]
    th = api.sample_prior(3, S.TCM2_IRR, lo, hi, 5000)
    t = api.unit_box(th, 5000, 4, lo, hi).cpu().numpy()
    ref = (th.cpu().numpy()[:, :4] - np.asarray(lo)) / (np.asarray(hi) - np.asarray(lo))
    assert np.allclose(t, np.clip(ref, 0, 1), atol=1e-6) and t.min() >= 0 and t.max() <= 1
    # noise: y - x = l sigma z with l = q ||x|| / ||sigma||; chunked calls reproduce one call
    inp = S.feng_polyexp(*S.draw_feng(3))
    x = api.simulate(S.TCM2_IRR, ts, te, inp, th)
    yn = api.add_noise(x, ts, te, 109.8, 0.1, 0.1, 99)
    y2 = torch.empty_like(x)
    api.add_noise(x[:1234], ts, te, 109.8, 0.1, 0.1, 99, first_index=0, out=y2[:1234])
    api.add_noise(x[1234:], ts, te, 109.8, 0.1, 0.1, 99, first_index=1234, out=y2[1234:])
    assert torch.equal(yn[:, :L], y2[:, :L])
    xc = x.cpu().numpy()[:, :L].astype(np.float64)
    e = yn.cpu().numpy()[:, :L] - xc
    tm = 0.5 * (ts + te)
    sig = np.sqrt(np.maximum(xc, 0) * np.exp(np.log(2) / 109.8 * tm) / (te - ts))
    lvl = 0.1 * np.linalg.norm(xc, axis=1) / np.linalg.norm(sig, axis=1)
    ok = sig > 0
    z = e[ok] / (lvl[:, None] * sig)[ok]
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    # q = 0 leaves the TACs untouched
    y0 = api.add_noise(x, ts, te, 109.8, 0.0, 0.0, 7)
    assert torch.equal(y0[:, :L], x[:, :L])


def _philox_u01(orc, i, j, seed):
    r = orc.philox4x32_10([i, j & 0xFFFFFFFF, j >> 32, 0x4C4F43], [seed & 0xFFFFFFFF, seed >> 32])
    return ((r >> 9).astype(np.float64) + 0.5) * 2.0 ** -23


@pytest.fixture(scope="module")
def c3_small():
    from paper_2603_14859_b300 import synth as S
    from paper_2603_14859_b300.pipeline import make_y_gpu
    W = S.workload("totalbody_fdg", J=4096, N_per_model=1000)
    y = make_y_gpu(W)
    irr = np.nonzero(W.truth_model == S.TCM2_IRR)[0]
    truth = np.zeros((W.J, 4), np.float32)
    for th, rows in zip(W.truth, W.truth_rows):
        truth[rows] = th[:, :4]
    return W, y, irr, truth


@pytest.mark.parametrize("M,k", [(2000, 64), (10_000, 200)])
def test_local_abc_stage_parity(orc, c3_small, M, k):
    """Proposals, distances, accepted set, weights and summaries of the local
    kernel against the oracle fed the GPU's own proposals (M = 2000: selection
    over all distances; M = 10^4: over the candidates a pilot sample brackets)."""
    from paper_2603_14859_b300 import synth as S
    from paper_2603_14859_b300.learned import LearnedLocalAbc
    W, y, irr, truth = c3_small
    model = LearnedLocalAbc(W.ts, W.te, W.input_for(S.TCM2_IRR), W.half_life)
    L = W.L
    lo, hi = model.lo, model.hi
    rows = irr[:10]
    J = len(rows)
    rng = np.random.default_rng(8)
    u_true = (truth[rows].astype(np.float64) - lo) / (hi - lo)
    prop = np.zeros((J, 8), np.float32)
    prop[:, 0::2] = u_true + rng.normal(0, 0.05, u_true.shape)
    prop[:, 1::2] = np.log(rng.uniform(0.03, 0.3, u_true.shape))
    prop[0, 0::2] = [-0.5, 0.3, 1.4, 0.5]          # means outside the box on both sides
    yj = y[torch.from_numpy(rows).cuda()].contiguous()
    seed = 4242
    out = model.local(yj, torch.from_numpy(prop).cuda(), M=M, k=k, seed=seed, dump=True)
    u = out["u"].cpu().numpy().astype(np.float64)
    d = out["d"].cpu().numpy().astype(np.float64)
    yh = yj.cpu().numpy()[:, :L]
    w = model.w.astype(np.float64)
    mu = np.clip(prop[:, 0::2].astype(np.float64), -3, 4)
    sg = np.exp(np.clip(prop[:, 1::2].astype(np.float64), -7, 2))
    # (1) the sampler: inverse-CDF truncated normal of the Philox uniforms
    for j in range(J):
        for i in rng.choice(M, 40, replace=False):
            uu = _philox_u01(orc, int(i), int(j), seed)
            for p in range(4):
                ref = orc.truncnorm01(mu[j, p], sg[j, p], uu[p])
                assert abs(u[j, i, p] - ref) <= 2e-5 + 2e-5 * sg[j, p], (j, i, p, u[j, i, p], ref)
    n_sets_equal = 0
    for j in range(J):
        th = (lo + (hi - lo) * u[j]).astype(np.float32)
        x = orc.simulate(S.TCM2_IRR, W.ts, W.te, W.input_for(S.TCM2_IRR), th)
        dref = ((yh[j].astype(np.float64) - x) ** 2 * w).sum(1)
        yn = (w * yh[j].astype(np.float64) ** 2).sum()
        # (2) distances: table interpolation + fp32 arithmetic
        tol = 3e-5 * np.sqrt(dref * yn) + 1e-5 * dref
        assert np.all(np.abs(d[j] - dref) <= tol), np.abs(d[j] - dref).max()
        # (3) accepted set = k nearest of the oracle up to the near-tie band
        o = orc.local_abc(u[j], mu[j], sg[j], x, yh[j], w, k, lo, hi)
        gsel = np.lexsort((np.arange(M), d[j].astype(np.float32)))[:k]
        dk = np.sort(dref)[k - 1]
        diff = set(gsel.tolist()) ^ set(o["idx"].tolist())
        for i in diff:
            assert abs(dref[i] - dk) <= 2 * (3e-5 * np.sqrt(dk * yn) + 1e-5 * dk), (j, i)
        # (4) median accepted distance and ||y||_w^2
        assert float(out["dmed"][j]) == float(np.sort(d[j].astype(np.float32))[(k - 1) // 2])
        assert abs(float(out["ynorm"][j]) - yn) <= 1e-5 * yn
        if diff:
            continue
        n_sets_equal += 1
        # (5) weights and summaries on the same accepted set
        assert abs(float(out["ess"][j]) - o["ess"]) <= 1e-3 * o["ess"]
        vals = np.stack([lo[c] + (hi[c] - lo[c]) * u[j, o["idx"], c] for c in range(4)], 1)
        ki = vals[:, 0] * vals[:, 2] / (vals[:, 1] + vals[:, 2])
        vals = np.concatenate([vals, ki[:, None]], 1)
        for c in range(5):
            span = vals[:, c].max() - vals[:, c].min() + 1e-12
            assert abs(float(out["mean"][j, c]) - o["mean"][c]) <= 1e-4 * span + 1e-6 * abs(o["mean"][c])
            assert abs(float(out["sd"][j, c]) - o["sd"][c]) <= 1e-3 * o["sd"][c] + 1e-5 * span
            srt = np.sort(vals[:, c])
            for key, q in (("lo", o["lo"][c]), ("hi", o["hi"][c])):
                # the same order statistic, or its neighbour when fp32 weights cross the level differently
                gq = float(out[key][j, c])
                r_ref = int(np.argmin(np.abs(srt - q)))
                r_gpu = int(np.argmin(np.abs(srt - gq)))
                assert abs(gq - srt[r_gpu]) <= 1e-6 * abs(gq) + 1e-7 and abs(r_gpu - r_ref) <= 1
    assert n_sets_equal >= J - 2


def test_local_abc_edge_cases(c3_small):
    """k = M (everything accepted), k = 1, and ties broken by proposal index."""
    from paper_2603_14859_b300 import synth as S
    from paper_2603_14859_b300.learned import LearnedLocalAbc
    W, y, irr, truth = c3_small
    model = LearnedLocalAbc(W.ts, W.te, W.input_for(S.TCM2_IRR), W.half_life)
    yj = y[torch.from_numpy(irr[:3]).cuda()].contiguous()
    prop = LearnedLocalAbc.uniform_proposal(3)
    full = model.local(yj, prop, M=200, k=200, seed=1, dump=True)
    u = full["u"].cpu().numpy().astype(np.float64)
    vals = model.lo[None, None, :] + (model.hi - model.lo)[None, None, :] * u
    # near-flat proposal: equal-ish weights; the weighted mean is within the range of the values
    for c in range(4):
        m = full["mean"][:, c].cpu().numpy()
        assert np.all(m >= vals[:, :, c].min(1) - 1e-6) and np.all(m <= vals[:, :, c].max(1) + 1e-6)
    one = model.local(yj, prop, M=200, k=1, seed=1, dump=True)
    d = one["d"].cpu().numpy()
    best = d.argmin(1)
    ub = one["u"].cpu().numpy()[np.arange(3), best]
    th = model.lo + (model.hi - model.lo) * ub
    assert np.allclose(one["mean"][:, :4].cpu().numpy(), th, rtol=1e-6)
    assert np.all(one["sd"].cpu().numpy() == 0) and np.allclose(one["ess"].cpu().numpy(), 1.0)
    # degenerate proposal: means far below the box with sigma at its floor put every proposal on the
    # lower corner, so all distances tie; the accepted set is the lowest k indices, the posterior is
    # that corner and the weights are equal
    pt = torch.zeros((3, 8), device="cuda")
    pt[:, 0::2] = -3.0
    pt[:, 1::2] = -30.0
    for M in (700, 4096):     # 4096: the pilot bracket holds every distance and selection falls back
        tie = model.local(yj, pt, M=M, k=50, seed=2, dump=True)
        dd = tie["d"].cpu().numpy()
        assert np.all(tie["u"].cpu().numpy() == 0.0)
        assert np.all(dd == dd[:, :1])
        assert np.allclose(tie["mean"][:, :4].cpu().numpy(), model.lo.astype(np.float32), rtol=1e-6)
        assert np.all(tie["sd"].cpu().numpy() <= 1e-6)
        assert np.allclose(tie["ess"].cpu().numpy(), 50, rtol=1e-4)
        assert np.all(tie["dmed"].cpu().numpy() == dd[:, 0])


def test_training_is_bitwise_reproducible(c3_small):
    """Two trainings from the same seeds end with identical parameters (the
    weight-gradient GEMMs add their split-K partial sums in a fixed order)."""
    from paper_2603_14859_b300 import synth as S
    from paper_2603_14859_b300.learned import LearnedLocalAbc
    W = c3_small[0]
    ps = []
    for _ in range(2):
        model = LearnedLocalAbc(W.ts, W.te, W.input_for(S.TCM2_IRR), W.half_life, q_lo=0.1, q_hi=0.1)
        model.train(n_pairs=8192 * 40, batch=8192, log_every=0)
        ps.append(model.params.clone())
    assert torch.equal(ps[0], ps[1])


def test_learned_proposal_beats_prior_proposal(c3_small):
    """At the same draw budget per voxel, proposals from the trained network give
    posterior means much closer to the truth than prior-like proposals; the
    fallback routes voxels the local run cannot resolve to the global path."""
    from paper_2603_14859_b300 import synth as S
    from paper_2603_14859_b300.learned import GlobalIrr, LearnedLocalAbc, run_learned
    W, y, irr, truth = c3_small
    model = LearnedLocalAbc(W.ts, W.te, W.input_for(S.TCM2_IRR), W.half_life, q_lo=0.1, q_hi=0.1)
    log = model.train(n_pairs=10_000_000, batch=8192, log_every=20)
    first, last = log.losses[0][1], float(np.mean([l for _, l in log.losses[-5:]]))
    assert last < first - 3.0, log.losses
    rows = irr[:1024]
    yj = y[torch.from_numpy(rows).cuda()].contiguous()
    M, k = 10_000, 200
    learned = model.local(yj, model.propose(yj), M=M, k=k, seed=3)
    flat = model.local(yj, LearnedLocalAbc.uniform_proposal(len(rows)), M=M, k=k, seed=3)
    ut = (truth[rows].astype(np.float64) - model.lo) / (model.hi - model.lo)

    ki = truth[rows, 0].astype(np.float64) * truth[rows, 2] / (truth[rows, 1] + truth[rows, 2])

    def err(o):
        m = (o["mean"][:, :4].cpu().numpy().astype(np.float64) - model.lo) / (model.hi - model.lo)
        e = list(np.sqrt(((m - ut) ** 2).mean(0)))
        return np.array(e + [np.sqrt(((o["mean"][:, 4].cpu().numpy() - ki) ** 2).mean()) / ki.std()])

    el, ef = err(learned), err(flat)
    # K1, Vb and K_i are identified by the data and must gain; k2 and k3 barely are (the global
    # path's own error on them is ~0.35 of the box), so for those only require no loss.  With
    # these seeds (training is bitwise reproducible) the ratios are 0.22, 0.67, 0.99, 0.54, 0.90
    assert el[0] < 0.5 * ef[0] and el[3] < 0.8 * ef[3] and el[4] < 0.95 * ef[4], (el, ef)
    assert el[1] < 1.05 * ef[1] and el[2] < 1.05 * ef[2], (el, ef)
    # fallback: with a calibrated threshold, voxels whose local run is unreliable take the global path
    g = GlobalIrr(model, N=200_000, k=k)
    rel = g.calibrate(yj[:128])
    out, fb = run_learned(model, yj, M, k, g, rel)
    # the fallback takes exactly the voxels with few effective samples (or a NaN ESS) or a
    # large accepted distance, ascending
    bad = ~(out["ess"] >= k / 4) | (out["dmed"] > rel * out["ynorm"])
    assert torch.equal(torch.nonzero(bad).flatten().to(torch.int32), fb)
    if fb.numel():
        ref = g.run(yj.index_select(0, fb).contiguous())
        assert torch.equal(out["mean"].index_select(0, fb), ref["mean"])

"""Model probabilities and posterior summaries on the GPU against the oracle,
given the same accepted indices (Sec. II-D, Sec. III-B)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 2, 37, 200, 500])
def test_select_and_summaries(orc, k):
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(k)
    N = 4000
    off = [0, 1500, 4000]
    theta = rng.uniform(0.001, 1.0, (N, 8)).astype(np.float32)
    theta[:1500, 4:] = 0
    theta[1500:, 5:] = 0
    J = 333
    idx = np.stack([rng.choice(N, k, replace=False) for _ in range(J)]).astype(np.int32)
    idx[0] = np.arange(k)                       # all from model 0
    if k % 2 == 0:
        idx[1] = np.concatenate([np.arange(k // 2), 1500 + np.arange(k // 2)])   # exact 50/50 split
    ti, tt = torch.from_numpy(idx).cuda(), torch.from_numpy(theta).cuda()
    prob, pref = api.model_select(ti, off)
    op, opref = orc.model_select(idx, off)
    assert np.array_equal(pref.cpu().numpy(), opref)
    assert np.allclose(prob.cpu().numpy(), op, rtol=0, atol=1e-7)
    nparams, has_ki = [4, 5], [1, 1]
    g = api.summarize(tt, off, nparams, has_ki, [0, 1, 2], ti, pref)
    o = orc.summarize(theta, off, nparams, has_ki, [0, 1, 2], idx, opref)
    for a, b in zip(g, o):
        a = a.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        m = ~np.isnan(b)
        assert np.all(np.abs(a[m] - b[m]) <= 1e-5 * np.abs(b[m]) + 1e-7)
    # all-draws summaries (no preferred model)
    g = api.summarize(tt, off, nparams, has_ki, [0, 1, 2], ti, None)
    o = orc.summarize(theta, off, nparams, has_ki, [0, 1, 2], idx, None)
    for a, b in zip(g, o):
        a = a.cpu().numpy().astype(np.float64)
        m = ~np.isnan(b)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.all(np.abs(a[m] - b[m]) <= 1e-5 * np.abs(b[m]) + 1e-7)


@pytest.mark.parametrize("shift", [0, 1])
def test_summaries_rows_on_and_off_alignment(orc, shift):
    """Parameter rows that start on a 16-byte boundary (read four values per load) and the
    same rows one element off it (read one value per load): the same summaries as the oracle,
    with and without a preferred model, for a k whose accepted rows fit the row table."""
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(4242 + shift)
    N, k, J = 4000, 200, 129
    off = [0, 1500, 4000]
    theta = rng.uniform(0.001, 1.0, (N, 8)).astype(np.float32)
    theta[:1500, 4:] = 0
    theta[1500:, 5:] = 0
    idx = np.stack([rng.choice(N, k, replace=False) for _ in range(J)]).astype(np.int32)
    flat = torch.zeros(N * 8 + shift, dtype=torch.float32, device="cuda")
    tt = flat[shift:].view(N, 8)
    tt.copy_(torch.from_numpy(theta))
    ti = torch.from_numpy(idx).cuda()
    _, pref = api.model_select(ti, off)
    _, opref = orc.model_select(idx, off)
    nparams, has_ki = [4, 5], [1, 1]
    for pr, opr in ((pref, opref), (None, None)):
        g = api.summarize(tt, off, nparams, has_ki, [0, 1, 2], ti, pr)
        o = orc.summarize(theta, off, nparams, has_ki, [0, 1, 2], idx, opr)
        for a, b in zip(g, o):
            a = a.cpu().numpy().astype(np.float64)
            assert np.array_equal(np.isnan(a), np.isnan(b))
            m = ~np.isnan(b)
            assert np.all(np.abs(a[m] - b[m]) <= 1e-5 * np.abs(b[m]) + 1e-7)


@pytest.mark.parametrize("k", [40, 200, 256, 300])
def test_summaries_with_many_ties(orc, k):
    """Parameter values from five distinct levels, so every order statistic of the 95 %
    interval falls inside a run of equal values; accepted counts per model on both sides of
    256 (the register tournament of the interval's order statistics handles 33 to 256
    values, the histogram selection the rest)."""
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(900 + k)
    N = 5000
    off = [0, 2000, 5000]
    theta = (rng.integers(1, 6, (N, 8)) / 5.0).astype(np.float32)
    J = 97
    idx = np.stack([rng.choice(N, k, replace=False) for _ in range(J)]).astype(np.int32)
    idx[0] = np.arange(k)                              # all from model 0
    ti, tt = torch.from_numpy(idx).cuda(), torch.from_numpy(theta).cuda()
    _, pref = api.model_select(ti, off)
    _, opref = orc.model_select(idx, off)
    nparams, has_ki = [4, 5], [1, 1]
    for pr, opr in ((pref, opref), (None, None)):
        g = api.summarize(tt, off, nparams, has_ki, [0, 1, 2], ti, pr)
        o = orc.summarize(theta, off, nparams, has_ki, [0, 1, 2], idx, opr)
        for a, b in zip(g, o):
            a = a.cpu().numpy().astype(np.float64)
            assert np.array_equal(np.isnan(a), np.isnan(b))
            m = ~np.isnan(b)
            assert np.all(np.abs(a[m] - b[m]) <= 1e-5 * np.abs(b[m]) + 1e-7)


@pytest.mark.parametrize("k,shift", [(64, 0), (64, 1), (2048, 0), (203, 0)])
def test_model_select_many_models(orc, k, shift):
    """Five models with uneven draw counts (one of them a single draw), index rows that
    start on and off a 16-byte boundary, k from 64 to the largest (2048) and k not a
    multiple of 4: every count equals the oracle's, ties going to the lower model."""
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(k + 7 * shift)
    off = [0, 10, 400, 3000, 3001, 9000]
    N = off[-1]
    J = 257
    idx = rng.integers(0, N, (J, k)).astype(np.int32)
    idx[0] = 3000                                       # every draw from the one-draw model
    idx[1, : k // 2], idx[1, k // 2:] = 5, 405          # a tie between models 0 and 2 (k even)
    flat = torch.zeros(J * k + shift, dtype=torch.int32, device="cuda")
    ti = flat[shift:].view(J, k)
    ti.copy_(torch.from_numpy(idx))
    prob, pref = api.model_select(ti, off)
    op, opref = orc.model_select(idx, off)
    assert np.array_equal(pref.cpu().numpy(), opref)
    assert np.allclose(prob.cpu().numpy(), op, rtol=0, atol=1e-7)


@pytest.mark.parametrize("k,P", [(2048, 30), (777, 12)])
def test_summaries_wide_rows(orc, k, P):
    """Many parameters at the largest k (every column's values fill the shared-memory
    buffer the order statistics use)."""
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(k + P)
    N = 6000
    off = [0, 2500, 6000]
    ld = P + 2
    theta = rng.gamma(2.0, 0.3, (N, ld)).astype(np.float32)
    J = 23
    idx = np.stack([rng.choice(N, k, replace=False) for _ in range(J)]).astype(np.int32)
    ti, tt = torch.from_numpy(idx).cuda(), torch.from_numpy(theta).cuda()
    _, pref = api.model_select(ti, off)
    _, opref = orc.model_select(idx, off)
    nparams, has_ki = [P - 3, P], [0, 1]
    for pr, opr in ((pref, opref), (None, None)):
        g = api.summarize(tt, off, nparams, has_ki, [1, 4, 2], ti, pr)
        o = orc.summarize(theta, off, nparams, has_ki, [1, 4, 2], idx, opr)
        for a, b in zip(g, o):
            a = a.cpu().numpy().astype(np.float64)
            assert a.shape == (J, P + 1)
            assert np.array_equal(np.isnan(a), np.isnan(b))
            m = ~np.isnan(b)
            assert np.all(np.abs(a[m] - b[m]) <= 1e-5 * np.abs(b[m]) + 1e-7)


@pytest.mark.parametrize("k", [1, 7, 200, 500, 2048])
def test_response_band(orc, k):
    """Posterior band of the lp-ntPET response function 1 + (gamma / k2a) g(t)
    against the oracle: draws of another model and padding (-1) are skipped, a voxel
    with no accepted lp-ntPET draw gives NaN, gamma = 0 gives exactly 1."""
    from paper_2603_14859_b300 import api
    from paper_2603_14859_b300 import synth as S
    rng = np.random.default_rng(100 + k)
    lo_p, hi_p = S.PRIORS[S.LPNTPET]
    n_other, n_lp = 3000, 5000
    th = np.zeros((n_other + n_lp, 8), np.float32)
    th[:n_other, :3] = rng.uniform(0.1, 1.0, (n_other, 3))
    th[n_other:, :7] = rng.uniform(lo_p, hi_p, (n_lp, 7))
    th[n_other:n_other + 500, 3] = 0.0                           # no activation
    first, last = n_other, n_other + n_lp
    J = 97
    idx = rng.integers(0, n_other + n_lp, (J, k)).astype(np.int32)
    idx[0] = rng.integers(0, n_other, k)                         # nothing from lp-ntPET
    idx[1] = n_other + rng.integers(0, 500, k)                   # only gamma = 0 draws
    if k > 3:
        idx[2, ::3] = -1
    ts = np.concatenate([[0.0, 19.5], np.linspace(20.0, 60.0, 17), [float(th[n_other + 7, 4]),
                                                                     float(th[n_other + 7, 4] + th[n_other + 7, 5])]])
    ts = ts.astype(np.float32)
    g = api.response_cri(torch.from_numpy(th).cuda(), first, last, ts, torch.from_numpy(idx).cuda())
    o = orc.response_cri(th, first, last, ts.astype(np.float64), idx)
    for a, b in zip(g, o):
        a = a.cpu().numpy().astype(np.float64)
        assert a.shape == (J, len(ts))
        assert np.array_equal(np.isnan(a), np.isnan(b))
        m = ~np.isnan(b)
        assert np.all(np.abs(a[m] - b[m]) <= 1e-5 * np.maximum(1.0, np.abs(b[m])) + 1e-6)
    assert np.all(np.isnan(g[0][0].cpu().numpy()))
    for a in g:
        assert np.all(a[1].cpu().numpy() == 1.0)

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


@pytest.mark.parametrize("k,P", [(2048, 30), (777, 12)])
def test_summaries_wide_rows(orc, k, P):
    """Many parameters at the largest k (the rows' columns are gathered in groups when
    one voxel's columns do not fit in shared memory together)."""
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

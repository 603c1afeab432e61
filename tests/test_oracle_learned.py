"""Pins for the oracle's learned-proposal functions (a build extra with no
paper counterpart): normal CDF / quantile, truncated normal, the MLP's
forward pass and analytic gradient, and importance-weighted local ABC."""
import math

import numpy as np
import pytest
from scipy import special, stats


def test_phi_and_quantile_against_scipy(orc):
    for z in [-8.0, -3.1, -1.0, 0.0, 0.3, 2.5, 7.9]:
        assert orc.Phi(z) == pytest.approx(special.ndtr(z), rel=1e-13, abs=1e-300)
    for p in [1e-12, 1e-6, 0.01, 0.3, 0.5, 0.77, 0.999, 1 - 1e-9]:
        assert orc.Phi_inv(p) == pytest.approx(special.ndtri(p), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("mu,sigma", [(0.5, 0.1), (0.05, 0.02), (1.3, 0.2), (-0.4, 0.5), (0.5, 30.0)])
def test_truncnorm_inverse_cdf_and_density(orc, mu, sigma):
    a, b = -mu / sigma, (1 - mu) / sigma
    dist = stats.truncnorm(a, b, loc=mu, scale=sigma)
    for u in [1e-6, 0.1, 0.5, 0.9, 0.999999]:
        t = orc.truncnorm01(mu, sigma, u)
        assert 0.0 <= t <= 1.0
        assert dist.cdf(t) == pytest.approx(u, rel=1e-7, abs=1e-9)
        assert orc.truncnorm01_logpdf(mu, sigma, t) == pytest.approx(dist.logpdf(t), rel=1e-9, abs=1e-9)


def _rand_params(D, H, O, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(size=H * D + H + H * H + H + O * H + O) * scale


def test_mlp_forward_one_unit_closed_form(orc):
    # D = H = 1, O = 2: out = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3
    D, H, O = 1, 1, 2
    W1, b1, W2, b2, W3, b3 = 0.7, -0.2, 1.3, 0.1, [0.5, -1.5], [0.05, 0.2]
    prm = np.array([W1, b1, W2, b2] + W3 + b3)
    gelu = lambda z: z * special.ndtr(z)
    x = np.array([[0.9], [-2.0]])
    out = orc.mlp_forward(prm, D, H, O, x)
    for n in range(2):
        h2 = gelu(W2 * gelu(W1 * x[n, 0] + b1) + b2)
        assert out[n].tolist() == pytest.approx([W3[0] * h2 + b3[0], W3[1] * h2 + b3[1]], rel=1e-14)


def test_mlp_gradient_against_finite_differences(orc):
    D, H, P = 5, 7, 2
    O = 2 * P
    prm = _rand_params(D, H, O, seed=3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(6, D))
    T = rng.uniform(0.02, 0.98, size=(6, P))
    loss, g = orc.mlp_loss_grad(prm, D, H, P, X, T)
    assert np.isfinite(loss)
    eps = 1e-6
    for i in rng.choice(len(prm), 40, replace=False):
        e = np.zeros_like(prm)
        e[i] = eps
        fd = (orc.mlp_loss_grad(prm + e, D, H, P, X, T)[0] - orc.mlp_loss_grad(prm - e, D, H, P, X, T)[0]) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=2e-5, abs=1e-8)


def test_mlp_loss_matches_truncnorm_nll(orc):
    D, H, P = 3, 4, 2
    prm = _rand_params(D, H, 2 * P, seed=9, scale=0.2)
    X = np.random.default_rng(1).normal(size=(3, D))
    T = np.array([[0.2, 0.7], [0.5, 0.5], [0.9, 0.1]])
    out = orc.mlp_forward(prm, D, H, 2 * P, X)
    ref = 0.0
    for n in range(3):
        for p in range(P):
            mu = np.clip(out[n, 2 * p], -3, 4)
            sg = math.exp(np.clip(out[n, 2 * p + 1], -7, 2))
            ref -= stats.truncnorm(-mu / sg, (1 - mu) / sg, loc=mu, scale=sg).logpdf(T[n, p])
    assert orc.mlp_loss_grad(prm, D, H, P, X, T)[0] == pytest.approx(ref / 3, rel=1e-10)


def test_local_abc_uniform_proposal_is_plain_abc(orc):
    """A very wide proposal gives equal weights: plain rejection-ABC summaries."""
    rng = np.random.default_rng(0)
    M, P, L, k = 400, 3, 6, 25
    u = rng.uniform(size=(M, P))
    x = rng.normal(size=(M, L))
    y = rng.normal(size=L).astype(np.float32)
    w = np.full(L, 1 / L)
    lo, hi = np.array([0.1, 0.2, 0.3]), np.array([1.0, 2.0, 0.5])
    r = orc.local_abc(u, [0.5] * P, [1e4] * P, x, y, w, k, lo, hi)
    d = ((y.astype(np.float64) - x) ** 2 * w).sum(1)
    acc = np.argsort(d, kind="stable")[:k]
    assert sorted(r["idx"].tolist()) == sorted(acc.tolist())
    th = lo + (hi - lo) * u[acc]
    assert r["ess"] == pytest.approx(k, rel=1e-6)
    assert np.allclose(r["mean"][:P], th.mean(0), rtol=1e-6)
    assert np.allclose(r["sd"][:P], th.std(0), rtol=1e-5)
    ki = th[:, 0] * th[:, 2] / (th[:, 1] + th[:, 2])
    assert r["mean"][P] == pytest.approx(ki.mean(), rel=1e-6)


def test_local_abc_importance_weights(orc):
    rng = np.random.default_rng(5)
    M, P, L, k = 300, 2, 4, 30
    mu, sg = np.array([0.3, 0.6]), np.array([0.1, 0.2])
    u = np.array([[orc.truncnorm01(mu[p], sg[p], rng.uniform()) for p in range(P)] for _ in range(M)])
    x = rng.normal(size=(M, L))
    y = rng.normal(size=L).astype(np.float32)
    w = np.full(L, 0.25)
    lo, hi = np.zeros(P), np.ones(P)
    r = orc.local_abc(u, mu, sg, x, y, w, k, lo, hi, ki=False)
    acc = r["idx"]
    q = np.prod([stats.truncnorm(-mu[p] / sg[p], (1 - mu[p]) / sg[p], loc=mu[p], scale=sg[p]).pdf(u[acc, p])
                 for p in range(P)], axis=0)
    W = (1 / q) / (1 / q).sum()
    assert r["mean"] == pytest.approx((W[:, None] * u[acc]).sum(0), rel=1e-9)
    assert r["ess"] == pytest.approx(1 / (W**2).sum(), rel=1e-9)

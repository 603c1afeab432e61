"""Pins for the oracle's TAC simulator (Sec. II-A, Eq. 1-4; Sec. III-A input).

Each check ties the oracle to something other than itself: a library ODE
solver, a closed-form integral, a mass balance, or an identity between models.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from paper_2603_14859_b300 import synth as S


def feng_value(beta, kappa, t):
    b1, b2, b3 = beta
    k1, k2, k3 = kappa
    return (b1 * t - b2 - b3) * math.exp(-k1 * t) + b2 * math.exp(-k2 * t) + b3 * math.exp(-k3 * t)


@pytest.fixture(scope="module")
def feng():
    beta, kap = S.draw_feng(1001)
    return beta, kap, S.feng_polyexp(beta, kap)


def test_feng_input_zero_at_origin_and_formula(orc, feng):
    beta, kap, cp = feng
    th = [0.5, 1.0, 0.1, 1.0]           # Vb = 1: the measured curve is the input itself
    assert abs(orc.tac_point(S.TCM2_IRR, th, cp, 0.0)) < 1e-9 * beta[1]
    for t in [0.001, 0.01, 0.3, 2.0, 40.0]:
        v = orc.tac_point(S.TCM2_IRR, th, cp, t)
        assert v == pytest.approx(feng_value(beta, kap, t), rel=1e-13)


@pytest.mark.parametrize("m", [0, 1, 2])
@pytest.mark.parametrize("d", [-2.5, -0.3, -1e-7, 0.0, 1e-9, 3e-4, 0.7, 5.0, 900.0])
@pytest.mark.parametrize("t", [0.01, 1.0, 47.0])
def test_Em_against_quadrature(orc, m, d, t):
    ref, _ = quad(lambda u: u**m * math.exp(-d * u), 0.0, t, epsabs=0, epsrel=1e-13, limit=200)
    assert orc.Em(m, d, t) == pytest.approx(ref, rel=1e-11)


def ode_frames(th, model, cpf, ts, te):
    """Frame means of Eq. 1-2 by a library ODE solver (DOP853), frame integrals as states."""
    if model == S.TCM2_IRR:
        K1, k2, k3, Vb = th
        k4 = 0.0
    else:
        K1, k2, k3, k4, Vb = th

    def f(t, y):
        cf, cm = y[0], y[1]
        c = cpf(t)
        return [K1 * c - (k2 + k3) * cf + k4 * cm, k3 * cf - k4 * cm, cf + cm, c]

    edges = np.concatenate([[0.0], te])
    sol = solve_ivp(f, [0, te[-1]], [0, 0, 0, 0], method="DOP853", rtol=1e-12, atol=1e-9, t_eval=edges,
                    first_step=1e-6, max_step=0.5)
    F = (1 - Vb) * sol.y[2] + Vb * sol.y[3]
    return np.diff(F) / np.diff(edges)


@pytest.mark.parametrize("model", [S.TCM2_IRR, S.TCM2_REV])
def test_2tcm_closed_form_matches_ode(orc, feng, model):
    beta, kap, cp = feng
    ts, te = S.frames_brain_fdg22()
    rows = [[0.5, 1.2, 0.1, 0.0, 0.05], [0.8, 0.3, 0.25, 0.05, 0.1], [0.2, 0.05, 0.001, 0.1, 0.2],
            # k2 + k3 on top of the input rate kappa2: the near-degenerate convolution
            [0.6, float(kap[1]) - 0.2, 0.2, 0.02, 0.1], [0.6, float(kap[1]) - 0.2 + 1e-7, 0.2, 0.0, 0.1]]
    th = np.array(rows, np.float32)
    if model == S.TCM2_IRR:
        th = th[:, [0, 1, 2, 4]]
    x = orc.simulate(model, ts, te, cp, th)
    cpf = lambda t: feng_value(beta, kap, t)
    for r in range(len(th)):
        ref = ode_frames([float(v) for v in th[r]], model, cpf, ts, te)
        assert np.max(np.abs(x[r] - ref) / np.abs(ref)) < 1e-9


def test_2tcm_mass_balance(orc, feng):
    """Reversible 2TCM with Vb = 0: int_0^inf C_T = (K1/k2)(1 + k3/k4) int_0^inf C_p."""
    beta, kap, cp = feng
    b1, b2, b3 = beta
    k1, k2_, k3_ = kap
    auc_p = b1 / k1**2 - (b2 + b3) / k1 + b2 / k2_ + b3 / k3_
    K1, k2, k3, k4 = 0.6, 0.4, 0.2, 0.1
    th = np.array([[K1, k2, k3, k4, 0.0]], np.float32)
    K1, k2, k3, k4 = [float(v) for v in th[0, :4]]
    T = 9000.0                      # slowest rate >= 0.01/min: tail below 1e-30
    x = orc.simulate(S.TCM2_REV, [0.0], [T], cp, th)
    assert x[0, 0] * T == pytest.approx(K1 / k2 * (1 + k3 / k4) * auc_p, rel=1e-10)


def test_2tcm_irreversible_plateau_is_Ki_times_auc(orc, feng):
    """k4 = 0: C_T(inf) = C_m(inf) = K_i int_0^inf C_p with K_i = K1 k3/(k2 + k3) (Sec. III-B)."""
    beta, kap, cp = feng
    b1, b2, b3 = beta
    k1, k2_, k3_ = kap
    auc_p = b1 / k1**2 - (b2 + b3) / k1 + b2 / k2_ + b3 / k3_
    th = np.array([0.7, 0.9, 0.3, 0.0], np.float32)
    K1, k2, k3 = [float(v) for v in th[:3]]
    v = orc.tac_point(S.TCM2_IRR, th, cp, 9000.0)
    assert v == pytest.approx(K1 * k3 / (k2 + k3) * auc_p, rel=1e-12)


def test_mrtm_equals_one_tissue_target_over_reference(orc, feng):
    """Target 1TC(K1, k2a) and reference 1TC(K1', k2'): MRTM with R1 = K1/K1', k2 = R1 k2'
    reproduces the target TAC (Eq. 3 with gamma = 0)."""
    beta, kap0, _ = feng
    beta, kap = S.draw_feng(1002, avoid=[S.REF_K2])
    cp = S.feng_polyexp(beta, kap)
    cr = S.reference_tissue_polyexp(cp)
    ts, te = S.frames_raclopride60()
    R1, BP = np.float32(1.3), np.float32(1.5)
    k2 = np.float32(float(R1) * S.REF_K2)
    k2a = float(k2) / (1.0 + float(BP))
    K1 = float(R1) * S.REF_K1
    x_m = orc.simulate(S.MRTM, ts, te, cr, np.array([[R1, k2, BP]], np.float32))
    # the target as a 2TCM with k3 = k4 = Vb = 0 is exactly a 1-tissue model
    x_t = orc.simulate(S.TCM2_REV, ts, te, cp, np.array([[K1, k2a, 0.0, 0.0, 0.0]], np.float32))
    # float32 rounding of K1 and k2a enters both sides differently: compare at 1e-6
    assert np.max(np.abs(x_m - x_t) / np.abs(x_t)) < 2e-6


@pytest.fixture(scope="module")
def racl():
    beta, kap = S.draw_feng(1002, avoid=[S.REF_K2])
    cr = S.reference_tissue_polyexp(S.feng_polyexp(beta, kap))
    ts, te = S.frames_raclopride60()
    return cr, ts, te


def test_lpntpet_gamma0_equals_mrtm(orc, racl):
    cr, ts, te = racl
    th_l = np.array([[1.1, 0.3, 2.0, 0.0, 30.0, 5.0, 1.0], [0.7, 0.55, 0.2, 0.0, 22.0, 2.0, 3.0]], np.float32)
    x_l = orc.simulate(S.LPNTPET, ts, te, cr, th_l)
    x_m = orc.simulate(S.MRTM, ts, te, cr, th_l[:, :3].copy())
    assert np.max(np.abs(x_l - x_m) / np.abs(x_m)) < 1e-8


def test_lpntpet_step_activation_equals_piecewise_mrtm(orc, racl):
    """alpha = 0 makes g a unit step at t_D: after t_D the model is MRTM with
    k2a -> k2a + gamma, started from the MRTM state at t_D (closed form)."""
    cr, ts, te = racl
    th = np.array([1.2, 0.4, 1.0, 0.15, 33.0, 5.0, 0.0], np.float32)
    R1, k2, BP, gam, tD = [float(v) for v in th[:5]]
    k2a = k2 / (1 + BP)
    a = k2a + gam

    def crv(t):
        return orc.tac_point(S.MRTM, [1.0, 0.0, 0.0], cr, t)        # R1 = 1, k2 = 0 -> C_r

    def conv(rate, t):                                             # (C_r conv exp(-rate t))(t)
        return orc.tac_point(S.MRTM, [0.0, rate, 0.0], cr, t) / rate

    zD = (k2 - R1 * k2a) * conv(k2a, tD)

    def C(t):
        if t < tD:
            return R1 * crv(t) + (k2 - R1 * k2a) * conv(k2a, t)
        z = math.exp(-a * (t - tD)) * zD + (k2 - R1 * a) * (conv(a, t) - math.exp(-a * (t - tD)) * conv(a, tD))
        return R1 * crv(t) + z

    ref = []
    for s, e in zip(ts, te):
        pts = [tD] if s < tD < e else None
        v, _ = quad(C, s, e, points=pts, epsabs=0, epsrel=1e-12, limit=200)
        ref.append(v / (e - s))
    x = orc.simulate(S.LPNTPET, ts, te, cr, th[None, :])
    assert np.max(np.abs(x[0] - ref) / np.abs(ref)) < 1e-8


def test_gamma_variate_shape(orc):
    assert orc.gamma_variate(10.0, 20.0, 25.0, 2.0) == 0.0
    assert orc.gamma_variate(25.0, 20.0, 25.0, 2.0) == pytest.approx(1.0)       # peak 1 at t_P
    # maximum of x^a exp(a(1-x)) is at x = 1
    xs = np.linspace(20.01, 60, 2000)
    g = [orc.gamma_variate(t, 20.0, 25.0, 2.0) for t in xs]
    assert abs(xs[int(np.argmax(g))] - 25.0) < 0.05


def test_gauss_legendre_nodes_exact_on_polynomials(orc):
    x, w = orc.gl_nodes()
    for deg in range(0, 40):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert (w * x**deg).sum() == pytest.approx(exact, abs=1e-14)


def _lp_rows(rng, n, gamma=None):
    """lp-ntPET parameter rows (R1, k2, BP_ND, gamma, t_D, t_P - t_D, alpha) inside the priors."""
    lo, hi = S.PRIORS[S.LPNTPET]
    th = rng.uniform(lo, hi, (n, 7)).astype(np.float32)
    if gamma is not None:
        th[:, 3] = gamma
    return th


def test_response_band_flat_without_activation(orc):
    """gamma = 0 leaves k2a(t) = k2a: the band is the constant 1 at every time."""
    rng = np.random.default_rng(11)
    th = _lp_rows(rng, 300, gamma=0.0)
    idx = rng.integers(0, 300, (5, 40)).astype(np.int32)
    mean, lo, hi = orc.response_cri(th, 0, 300, np.linspace(0, 60, 13), idx)
    assert np.all(mean == 1.0) and np.all(lo == 1.0) and np.all(hi == 1.0)


def test_response_band_before_onset_and_at_peak(orc):
    """Before every t_D the response is 1; one accepted draw at its own t_P gives
    1 + gamma / k2a = 1 + gamma (1 + BP_ND) / k2 (g(t_P) = 1)."""
    rng = np.random.default_rng(12)
    th = _lp_rows(rng, 50)
    idx = np.arange(50, dtype=np.int32).reshape(5, 10)
    mean, lo, hi = orc.response_cri(th, 0, 50, [0.0, 5.0, float(th[:, 4].min()) - 1e-3], idx)
    assert np.all(mean == 1.0) and np.all(lo == 1.0) and np.all(hi == 1.0)
    for i in (0, 17, 49):
        r = th[i].astype(np.float64)
        tP = r[4] + r[5]
        m, a, b = orc.response_cri(th, 0, 50, [tP], np.array([[i]], np.int32))
        want = 1.0 + r[3] * (1.0 + r[2]) / r[1]
        assert m[0, 0] == pytest.approx(want, rel=1e-12) and a[0, 0] == m[0, 0] and b[0, 0] == m[0, 0]


def test_response_band_matches_direct_quantiles(orc):
    """Mean and type-7 quantiles against numpy on responses written from the closed
    form x^alpha exp(alpha (1 - x)), x = (t - t_D) / (t_P - t_D); draws outside
    [first, last) (the other model's) are ignored; none left gives NaN."""
    rng = np.random.default_rng(13)
    th = np.vstack([rng.uniform(0, 1, (400, 7)).astype(np.float32), _lp_rows(rng, 600)])
    first, last = 400, 1000
    idx = rng.integers(0, 1000, (6, 75)).astype(np.int32)
    idx[5] = rng.integers(0, 400, 75)                # no lp-ntPET draw accepted
    ts = np.array([21.0, 30.0, 37.5, 45.0, 59.0])
    mean, lo, hi = orc.response_cri(th, first, last, ts, idx)
    for j in range(5):
        rows = th[idx[j][(idx[j] >= first) & (idx[j] < last)]].astype(np.float64)
        for m, t in enumerate(ts):
            x = (t - rows[:, 4]) / rows[:, 5]
            g = np.where(x > 0, np.abs(x) ** rows[:, 6] * np.exp(rows[:, 6] * (1.0 - x)), 0.0)
            v = 1.0 + rows[:, 3] * (1.0 + rows[:, 2]) / rows[:, 1] * g
            assert mean[j, m] == pytest.approx(v.mean(), rel=1e-12)
            assert lo[j, m] == pytest.approx(np.quantile(v, 0.025), rel=1e-12, abs=1e-15)
            assert hi[j, m] == pytest.approx(np.quantile(v, 0.975), rel=1e-12, abs=1e-15)
    assert np.all(np.isnan(mean[5])) and np.all(np.isnan(lo[5])) and np.all(np.isnan(hi[5]))

"""Host-side reductions of the budget calibration (Sec. II-C): the U-curve fit, the
ROC AUC and the elbow, each against a closed form or brute force; plus a small
sweep over the GPU path."""
import itertools
import math

import numpy as np
import pytest

from paper_2603_14859_b300 import calibrate as C


def test_u_curve_minimum_recovers_a_parabola_in_log_n():
    n = np.array([1e3, 3e3, 1e4, 3e4, 1e5, 3e5])
    u0 = math.log(2e4)
    mse = 0.7 + 0.05 * (np.log(n) - u0) ** 2
    best, (a, b, c) = C.u_curve_minimum(n, mse)
    assert best == pytest.approx(2e4, rel=1e-9)
    assert c == pytest.approx(0.05, rel=1e-9)


def test_u_curve_minimum_falls_back_to_the_grid():
    n = [1e3, 1e4, 1e5, 1e6]
    assert C.u_curve_minimum(n, [4.0, 3.0, 2.0, 1.0])[0] == 1e6          # decreasing: no interior minimum
    assert C.u_curve_minimum(n, [1.0, 3.0, 3.0, 1.5])[0] == 1e3          # opens downwards
    assert C.u_curve_minimum([10, 20], [2.0, 1.0])[0] == 20               # too few points to fit


def test_roc_auc_against_pairwise_counting():
    rng = np.random.default_rng(5)
    for _ in range(20):
        m = int(rng.integers(2, 40))
        s = rng.integers(0, 6, m).astype(float)                          # many ties
        y = rng.random(m) < 0.4
        if y.all() or not y.any():
            continue
        pos, neg = s[y], s[~y]
        brute = sum((a > b) + 0.5 * (a == b) for a, b in itertools.product(pos, neg)) / (len(pos) * len(neg))
        assert C.roc_auc(s, y) == pytest.approx(brute, abs=1e-12)
    assert C.roc_auc([0.1, 0.9], [0, 1]) == 1.0
    assert C.roc_auc([0.9, 0.1], [0, 1]) == 0.0
    assert math.isnan(C.roc_auc([0.3, 0.4], [1, 1]))


def test_elbow_of_a_saturating_curve():
    x = np.geomspace(1e3, 1e6, 13)
    y = 1.0 - np.exp(-x / 2e4)                 # rises, then flattens
    i = C.elbow(x, y)
    assert 1e4 <= x[i] <= 2e5
    assert C.elbow(x, np.linspace(0, 1, 13) ** 3) == 0      # convex in log x: never above its chord
    assert C.elbow(x, np.ones(13)) == 0


@pytest.mark.gpu
def test_small_sweeps_run_on_the_gpu_path():
    pts = C.mse_sweep([4000, 16000], k=40, J=256)
    for pt in pts:
        (vals,) = pt.mse.values()
        assert len(vals) == 4 and all(np.isfinite(v) and v >= 0 for v in vals)
    # more draws at a fixed k: the posterior means of K1 move closer to the truth
    assert pts[1].mse["2TCM-irr"][0] < pts[0].mse["2TCM-irr"][0]
    sel = C.selection_sweep([20000, 80000], k=100, J=1024)
    for pt in sel:
        assert 0.0 <= pt.accuracy <= 1.0 and 0.0 <= pt.auc <= 1.0


def test_poisson_noise_statistics():
    """y = Pois(l2 x) / l2 has mean x and variance x / l2 (checked on 200,000 draws
    per frame, within 5 standard errors), and never a negative value."""
    from paper_2603_14859_b300 import synth as S
    x = np.tile(np.array([[0.5, 2.0, 7.5]]), (200_000, 1))
    l2 = 3.0
    y = S.add_noise_poisson(x, l2, seed=9).astype(np.float64)
    m, v = y.mean(0), y.var(0)
    se_m = np.sqrt(x[0] / l2 / len(y))
    assert np.all(np.abs(m - x[0]) < 5 * se_m)
    assert np.all(np.abs(v / (x[0] / l2) - 1.0) < 0.02)
    assert y.min() >= 0.0
    # the scale puts the median voxel's expected relative noise at q
    xc = np.array([[1.0, 2.0, 3.0], [2.0, 2.0, 2.0], [4.0, 0.0, 4.0]])
    q = 0.1
    l2 = S.poisson_scale(xc, q)
    r = np.sqrt(xc.sum(1) / l2) / np.linalg.norm(xc, axis=1)
    assert np.median(r) == pytest.approx(q, rel=1e-12)


def test_detection_workload_shape():
    """61 one-minute frames, exactly half of the TACs activated (gamma >= 0.05)."""
    from paper_2603_14859_b300 import synth as S
    W = S.workload("raclopride_e2", J=400, N_per_model=1000, noise="poisson", level="low")
    assert W.L == 61 and np.allclose(W.te - W.ts, 1.0)
    act = W.truth_model == S.LPNTPET
    assert act.sum() == 200
    (th_m, th_a) = W.truth
    assert th_a.shape == (200, 7) and np.all(th_a[:, 3] >= 0.05)
    assert W.noise == "poisson" and W.noise_q == 0.03


@pytest.mark.gpu
def test_small_detection_sweep_on_the_gpu_path():
    pts = C.detection_sweep([20000], k=100, J=400)
    assert len(pts) == 4
    for pt in pts:
        assert 0.0 <= pt.sensitivity <= 1.0 and 0.0 <= pt.specificity <= 1.0 and 0.0 <= pt.auc <= 1.0

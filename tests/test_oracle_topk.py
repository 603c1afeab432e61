"""Pins for the oracle's distance + top-k (Algorithm 1, steps 4-5) and its
model selection / posterior summaries (Sec. II-D, Sec. III-B)."""
import numpy as np
import pytest


def rand_case(J=7, N=300, L=11, seed=0):
    rng = np.random.default_rng(seed)
    y = rng.normal(size=(J, L)).astype(np.float32)
    x = rng.normal(size=(N, L))
    w = rng.uniform(0.1, 1.0, L)
    return y, x, w / w.sum()


def test_topk_brute_force(orc):
    y, x, w = rand_case()
    k = 5
    idx, dist = orc.topk(y, x, w, k)
    for j in range(len(y)):
        d = [sum(w[l] * (float(y[j, l]) - x[n, l]) ** 2 for l in range(y.shape[1])) for n in range(len(x))]
        order = sorted(range(len(x)), key=lambda n: (d[n], n))[:k]
        assert idx[j].tolist() == order
        assert np.allclose(dist[j], [d[n] for n in order], rtol=1e-14)


def test_topk_k_equals_n_and_k_one(orc):
    y, x, w = rand_case(J=3, N=40)
    idx, dist = orc.topk(y, x, w, 40)
    assert all(sorted(r.tolist()) == list(range(40)) for r in idx)
    assert np.all(np.diff(dist, axis=1) >= 0)
    i1, d1 = orc.topk(y, x, w, 1)
    assert np.array_equal(i1[:, 0], idx[:, 0])


def test_noise_free_recovery(orc):
    y, x, w = rand_case(J=5, N=500)
    istar = [17, 0, 499, 250, 3]
    for j, i in enumerate(istar):
        x[i] = y[j].astype(np.float64)
    idx, dist = orc.topk(y, x, w, 3)
    assert idx[:, 0].tolist() == istar
    assert np.all(dist[:, 0] == 0.0)


def test_ties_go_to_lower_index(orc):
    y, x, w = rand_case(J=2, N=50)
    x[40] = x[7]
    x[9] = x[7]
    y[0] = x[7].astype(np.float32)
    x[[7, 9, 40]] = y[0].astype(np.float64)
    idx, _ = orc.topk(y, x, w, 3)
    assert idx[0].tolist() == [7, 9, 40]


def test_permutation_and_weight_scale_invariance(orc):
    y, x, w = rand_case(J=6, N=400, seed=3)
    idx, dist = orc.topk(y, x, w, 9)
    perm = np.random.default_rng(1).permutation(len(x))
    ip, dp = orc.topk(y, x[perm], w, 9)
    assert np.array_equal(perm[ip], idx)          # no exact ties in continuous random data
    i2, d2 = orc.topk(y, x, 3.0 * w, 9)
    assert np.array_equal(i2, idx)
    assert np.allclose(d2, 3.0 * dist, rtol=1e-14)
    vp = np.random.default_rng(2).permutation(len(y))
    iv, _ = orc.topk(y[vp], x, w, 9)
    assert np.array_equal(iv, idx[vp])


def test_model_select_counts_and_ties(orc):
    off = [0, 100, 250]
    idx = np.array([[1, 2, 101, 102], [150, 160, 170, 5], [0, 1, 2, 3], [120, 130, 140, 200]], np.int32)
    prob, pref = orc.model_select(idx, off)
    assert prob.tolist() == [[0.5, 0.5], [0.25, 0.75], [1.0, 0.0], [0.0, 1.0]]
    assert pref.tolist() == [0, 1, 0, 1]          # 50/50 -> first-listed (simpler) model
    p1, r1 = orc.model_select(idx[2:3], [0, 1000])
    assert p1.tolist() == [[1.0]] and r1.tolist() == [0]


def test_summary_against_textbook_statistics(orc):
    rng = np.random.default_rng(5)
    N = 1000
    theta = rng.uniform(0.01, 1.0, (N, 5)).astype(np.float32)
    off = [0, 600, 1000]                          # model 0: 2TCM-irr (4 params), model 1: 2TCM-rev (5)
    nparams, has_ki, ki_cols = [4, 5], [1, 1], [0, 1, 2]
    J, k = 6, 40
    idx = np.stack([rng.choice(N, k, replace=False) for _ in range(J)]).astype(np.int32)
    prob, pref = orc.model_select(idx, off)
    mean, sd, lo, hi = orc.summarize(theta, off, nparams, has_ki, ki_cols, idx, pref)
    for j in range(J):
        m = int(pref[j])
        sel = [i for i in idx[j] if off[m] <= i < off[m + 1]]
        th = theta[sel].astype(np.float64)
        P = nparams[m]
        ki = th[:, 0] * th[:, 2] / (th[:, 1] + th[:, 2])
        cols = [th[:, p] for p in range(P)]
        for p, v in enumerate(cols):
            assert mean[j, p] == pytest.approx(v.mean(), rel=1e-13)
            assert sd[j, p] == pytest.approx(v.std(ddof=1), rel=1e-12)
            q = np.quantile(v, [0.025, 0.975], method="linear")       # type 7
            assert lo[j, p] == pytest.approx(q[0], rel=1e-13) and hi[j, p] == pytest.approx(q[1], rel=1e-13)
        for p in range(P, 5):
            assert np.isnan(mean[j, p])
        assert mean[j, 5] == pytest.approx(ki.mean(), rel=1e-13)
        assert sd[j, 5] == pytest.approx(ki.std(ddof=1), rel=1e-12)


def test_summary_degenerate_cases(orc):
    theta = np.array([[0.5, 0.3, 0.2, 0.1], [0.5, 0.3, 0.2, 0.1], [0.9, 0.1, 0.4, 0.05]], np.float32)
    off = [0, 3]
    idx1 = np.array([[2]], np.int32)
    mean, sd, lo, hi = orc.summarize(theta, off, [4], [1], [0, 1, 2], idx1)
    t2 = theta[2].astype(np.float64)
    assert np.allclose(mean[0, :4], t2) and np.all(sd[0] == 0) and np.allclose(lo[0, :4], t2)
    assert mean[0, 4] == pytest.approx(t2[0] * t2[2] / (t2[1] + t2[2]), rel=1e-15)
    # K_i of (0.5, 0.3, 0.2): 0.5 * 0.2 / 0.5 = 0.2 (in float32 inputs)
    idx2 = np.array([[0, 1]], np.int32)
    mean, sd, lo, hi = orc.summarize(theta, off, [4], [1], [0, 1, 2], idx2)
    assert np.all(sd[0] == 0.0)
    assert mean[0, 4] == pytest.approx(0.2, rel=1e-7)


def test_summary_model_without_ki(orc):
    theta = np.random.default_rng(0).uniform(size=(20, 3)).astype(np.float32)
    idx = np.arange(10, dtype=np.int32)[None, :]
    mean, sd, lo, hi = orc.summarize(theta, [0, 20], [3], [0], [0, 1, 2], idx)
    assert np.isnan(mean[0, 3]) and np.isfinite(mean[0, :3]).all()


def test_l1_topk_brute_force_and_single_frame(orc):
    """L1 top-k (Sec. V): brute force on tiny inputs (sum_l w_l |y_l - x_l| written out
    per pair, then sorted by (distance, index)), and with one frame the order of
    |y - x| itself."""
    rng = np.random.default_rng(31)
    J, N, L, k = 5, 60, 7, 9
    y = rng.normal(size=(J, L)).astype(np.float32)
    x = rng.normal(size=(N, L))
    x[17] = x[3]                                   # an exact tie, broken by the index
    w = rng.uniform(0.1, 1.0, L)
    idx, dist = orc.topk_l1(y, x, w, k)
    for j in range(J):
        d = [sum(w[l] * abs(float(y[j, l]) - x[n, l]) for l in range(L)) for n in range(N)]
        order = sorted(range(N), key=lambda n: (d[n], n))[:k]
        assert list(idx[j]) == order
        assert np.allclose(dist[j], [d[n] for n in order], rtol=1e-14, atol=0)
    y1 = rng.normal(size=(3, 1)).astype(np.float32)
    x1 = rng.normal(size=(40, 1))
    idx1, d1 = orc.topk_l1(y1, x1, np.array([2.0]), 5)
    for j in range(3):
        assert list(idx1[j]) == list(np.argsort(np.abs(float(y1[j, 0]) - x1[:, 0]), kind="stable")[:5])
        assert np.allclose(d1[j], 2.0 * np.sort(np.abs(float(y1[j, 0]) - x1[:, 0]))[:5], rtol=1e-14)


def test_l1_distance_is_a_metric_and_differs_from_l2(orc):
    """The L1 distances satisfy the triangle inequality through a third point, and the
    L1 and squared-L2 orders differ on a case built for it (one large frame difference
    against many small ones)."""
    rng = np.random.default_rng(32)
    L = 6
    w = np.ones(L)
    y = rng.normal(size=(1, L)).astype(np.float32)
    x = rng.normal(size=(200, L))
    _, d_all = orc.topk_l1(y, x, w, 200)
    i_sorted, _ = orc.topk_l1(y, x, w, 200)
    dy = np.empty(200)
    dy[i_sorted[0]] = d_all[0]
    # d(y, x_n) <= d(y, x_0) + d(x_0, x_n) for every n (x_0 exactly representable)
    x[0] = x[0].astype(np.float32)
    _, d_0 = orc.topk_l1(x[:1].astype(np.float32), x, w, 200)
    i0, _ = orc.topk_l1(x[:1].astype(np.float32), x, w, 200)
    d0 = np.empty(200)
    d0[i0[0]] = d_0[0]
    assert np.all(dy <= dy[0] + d0 + 1e-12)
    yy = np.zeros((1, 4), np.float32)
    xx = np.array([[2.0, 0, 0, 0], [0.9, 0.9, 0.9, 0.9]])      # L1: 2.0 vs 3.6; squared L2: 4.0 vs 3.24
    i_l1, _ = orc.topk_l1(yy, xx, np.ones(4), 1)
    i_l2, _ = orc.topk(yy, xx, np.ones(4), 1)
    assert i_l1[0, 0] == 0 and i_l2[0, 0] == 1

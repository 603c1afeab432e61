"""Pins for the oracle's Philox4x32-10 and prior sampler (Algorithm 1, steps 1-2)."""
import os

import numpy as np

from paper_2603_14859_b300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert orc.philox4x32_10(ctr, key).tolist() == out


def test_prior_in_box_and_uniform(orc):
    lo, hi = S.PRIORS[S.TCM2_REV]
    th = orc.sample_prior(123, S.TCM2_REV, lo, hi, 200_000)
    assert th.dtype == np.float32 and th.shape == (200_000, 5)
    for p in range(5):
        v = th[:, p].astype(np.float64)
        assert v.min() >= np.float32(lo[p]) and v.max() <= np.float32(hi[p])
        u = (v - lo[p]) / (hi[p] - lo[p])
        # mean 1/2, variance 1/12 of U(0,1): 5-sigma bounds
        assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(u))
        assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / len(u))
    # parameters are not correlated with each other
    c = np.corrcoef(th.T.astype(np.float64))
    assert np.max(np.abs(c - np.eye(5))) < 0.02


def test_prior_counter_layout(orc):
    lo, hi = S.PRIORS[S.LPNTPET]
    a = orc.sample_prior(7, S.LPNTPET, lo, hi, 100)
    b = orc.sample_prior(7, S.LPNTPET, lo, hi, 40, first=60)
    assert np.array_equal(a[60:], b)
    # theta[n, p] comes from word p % 4 of counter (n, 0, model, p // 4)
    r = orc.philox4x32_10([5, 0, S.LPNTPET, 1], [7, 0])
    u = (int(r[1]) >> 8) * 2.0**-24
    assert a[5, 5] == np.float32(lo[5] + (hi[5] - lo[5]) * u)
    # different model id -> different stream
    c = orc.sample_prior(7, S.MRTM, lo[:3], hi[:3], 100)
    assert not np.array_equal(a[:, :3], c)

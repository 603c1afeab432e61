"""The learned path's reliability check in the library: the fallback predicate and
compaction, the row gather and scatter, and the device quantile that calibrates the
threshold, each against numpy / torch on the same inputs."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(J, seed):
    g = np.random.default_rng(seed)
    k = 200
    ess = g.uniform(0.0, 2.0 * k / 4, J).astype(np.float32)
    ess[g.random(J) < 0.01] = np.nan
    ess[g.random(J) < 0.01] = k / 4                      # exactly at the limit: reliable
    dmed = g.exponential(1.0, J).astype(np.float32)
    ynorm = g.uniform(5.0, 50.0, J).astype(np.float32)
    return k, ess, dmed, ynorm


@pytest.mark.parametrize("J", [1, 1000, 1024, 1025, 100_003])
@pytest.mark.parametrize("rel_max", [None, 0.05])
def test_fallback_rows_match_the_predicate(J, rel_max):
    from paper_2603_14859_b300 import api
    k, ess, dmed, ynorm = _case(J, J)
    t = [torch.from_numpy(a).cuda() for a in (ess, dmed, ynorm)]
    rows, count = api.fallback_rows(*t, k, rel_max)
    n = int(count.item())
    bad = ~(ess >= np.float32(k / 4))
    if rel_max is not None:
        bad |= dmed > np.float32(rel_max) * ynorm
    want = np.nonzero(bad)[0].astype(np.int32)
    assert n == want.size
    assert np.array_equal(rows[:n].cpu().numpy(), want)


def test_gather_and_scatter_rows():
    from paper_2603_14859_b300 import api
    J, W = 5000, 29
    k, ess, dmed, ynorm = _case(J, 7)
    rows, count = api.fallback_rows(*[torch.from_numpy(a).cuda() for a in (ess, dmed, ynorm)], k, 0.05)
    n = int(count.item())
    assert 0 < n < J
    src = torch.randn((J, 32), device="cuda")[:, :W]          # row stride 32 > width
    got = api.gather_rows(src, rows, count, n)
    idx = rows[:n].long()
    assert torch.equal(got, src.index_select(0, idx))
    dst = torch.zeros((J, 5), device="cuda")
    upd = torch.randn((n, 5), device="cuda")
    api.scatter_rows(upd, rows, count, dst)
    ref = torch.zeros((J, 5), device="cuda").index_copy_(0, idx, upd)
    assert torch.equal(dst, ref)
    # the count bounds the rows moved: entries past it are never touched
    zero = torch.zeros(1, dtype=torch.int32, device="cuda")
    dst2 = torch.full((J, 5), 7.0, device="cuda")
    api.scatter_rows(upd, rows, zero, dst2)
    assert bool((dst2 == 7.0).all())


@pytest.mark.parametrize("J,q", [(1, 0.5), (2, 0.99), (1000, 0.0), (1000, 1.0), (4097, 0.99), (100_000, 0.5),
                                 (100_000, 0.37)])
def test_median_rel_quantile_matches_numpy(J, q):
    """sum_l w_l y_l^2 = 1 exactly (one unit frame), so rel_j is the median column itself and
    the device selection must give numpy's quantile of those float32 values."""
    from paper_2603_14859_b300 import api
    g = np.random.default_rng(J)
    k, L = 9, 29
    dist = np.sort(g.exponential(1.0, (J, k)).astype(np.float32), axis=1)
    dist[g.random(J) < 0.05, (k - 1) // 2] = dist[0, (k - 1) // 2]    # ties
    y = np.zeros((J, L), np.float32)
    y[:, 3] = 1.0
    w = np.ones(L, np.float32)
    got = api.median_rel_quantile(torch.from_numpy(dist).cuda(), k, torch.from_numpy(y).cuda(), L, w, q)
    want = np.quantile(dist[:, (k - 1) // 2].astype(np.float64), q)
    assert got == pytest.approx(want, rel=1e-7, abs=0.0)

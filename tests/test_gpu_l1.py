"""Top-k by the frame-weighted L1 distance (Sec. V) on the GPU against the FP64
oracle: accepted sets equal up to the near-tie band, distances within the fp32
bound, ties to the lower draw index, and the list cuts exercised (N well above
the list capacity)."""
import numpy as np
import pytest
import torch

from parity import EPS32

pytestmark = pytest.mark.gpu


def _check(orc, y, x, w, k, idx, dist):
    L = y.shape[1]
    oi, od = orc.topk_l1(y, x.astype(np.float64), w.astype(np.float64), k)
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    tau = 4 * (L + 2) * EPS32
    for j in range(y.shape[0]):
        # distances of the GPU's own picks against fp64, and the sorted order
        d64 = (w[None, :].astype(np.float64) * np.abs(y[j].astype(np.float64)[None, :] - x[gi[j]])).sum(1)
        assert np.all(np.abs(gd[j] - d64) <= (L + 1) * EPS32 * d64 + 1e-30)
        assert np.all(np.diff(gd[j]) >= 0)
        same = gd[j][1:] == gd[j][:-1]
        assert np.all(gi[j][1:][same] > gi[j][:-1][same])          # equal distances: lower index first
        g, o = set(gi[j].tolist()), set(oi[j].tolist())
        if g != o:
            dk = od[j, -1]
            for n in g ^ o:
                dn = (w.astype(np.float64) * np.abs(y[j].astype(np.float64) - x[n])).sum()
                assert abs(dn - dk) <= tau * dk, (j, n, dn, dk)


@pytest.mark.parametrize("J,N,L,k", [(37, 3000, 22, 1), (64, 5000, 29, 50), (45, 2999, 60, 200), (9, 777, 7, 777)])
def test_l1_topk_against_oracle(orc, J, N, L, k):
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(J * 1000 + k)
    x = rng.gamma(2.0, 1.0, (N, L)).astype(np.float32)
    y = (x[rng.integers(0, N, J)] + rng.normal(0, 0.2, (J, L))).astype(np.float32)
    w = rng.uniform(0.2, 1.0, L).astype(np.float32)
    idx, dist = api.discrepancy_topk_l1(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda(), L, w, k)
    _check(orc, y, x, w, k, idx, dist)


def test_l1_ties_and_list_cuts(orc):
    """Many draws at exactly the same distance (duplicated rows) across the list cuts
    and the draw segments: the k kept are the lowest-index ones; with more ties than a
    list holds, the tie-overflow diagnostic counts the cuts that kept only the
    lowest-index ties (at least one per voxel)."""
    from paper_2603_14859_b300 import api
    rng = np.random.default_rng(77)
    L, k, N, J = 16, 20, 20000, 12
    base = rng.normal(size=(1, L)).astype(np.float32)
    y = np.repeat(base, J, 0)
    w = np.ones(L, np.float32)
    for stride, overflow in ((37, False), (2, True)):       # 541 ties (fit the lists), 10,000 (do not)
        x = rng.normal(size=(N, L)).astype(np.float32) * 3.0
        x[::stride] = base[0] + 0.5
        ws = torch.empty(api.l1_workspace_size(J, k), dtype=torch.uint8, device="cuda")
        idx, dist = api.discrepancy_topk_l1(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda(), L, w, k,
                                            workspace=ws)
        oi, od = orc.topk_l1(y[:1], x.astype(np.float64), w.astype(np.float64), k)
        assert np.array_equal(idx.cpu().numpy(), np.repeat(oi, J, 0))
        assert np.array_equal(oi[0], np.arange(k) * stride)
        st = api.l1_status(ws, J, k)
        assert (st >= J) if overflow else (st == 0)

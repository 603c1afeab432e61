"""Fused discrepancy + top-k (Algorithm 1 steps 4-5) against the FP64 oracle.

Stage parity: the oracle ranks the GPU's own simulated TACs, so any difference
is the discrepancy/top-k path alone.  Accepted sets must be identical except
for draws inside the near-tie band tau * d_(k), tau = 16 L eps32; returned
distances are the exact fp32 re-score (relative error <= 4 L eps32 vs fp64)."""
import numpy as np
import pytest
import torch

from paper_2603_14859_b300 import synth as S
from parity import check_topk_sets

pytestmark = pytest.mark.gpu


def _gpu_case(name, J, n, orc):
    from paper_2603_14859_b300 import api
    W = S.workload(name, J=J, N_per_model=n)
    # measured TACs from the oracle's simulator (no CUDA in the inputs)
    L = W.L
    xc = np.zeros((W.J, L))
    for th, rows in zip(W.truth, W.truth_rows):
        if len(rows):
            xc[rows] = orc.simulate(int(W.truth_model[rows[0]]), W.ts, W.te, W.inp, th)
    y = S.add_noise(xc, W.ts, W.te, W.half_life, W.q, W.z)
    ld = (L + 3) // 4 * 4
    yp = np.zeros((W.J, ld), np.float32)
    yp[:, :L] = y
    off = W.model_offsets()
    theta = torch.zeros((W.N, 8), device="cuda")
    x = torch.zeros((W.N, ld), device="cuda")
    for m, model in enumerate(W.models):
        lo, hi = W.priors(model)
        api.sample_prior(W.prior_seed, model, lo, hi, off[m + 1] - off[m], out=theta[off[m]:off[m + 1]])
        api.simulate(model, W.ts, W.te, W.inp, theta[off[m]:off[m + 1]], out=x[off[m]:off[m + 1]])
    return W, torch.from_numpy(yp).cuda(), x


def _compare(orc, W, y, x, k, prec, tau_extra=0.0, ws=None):
    from paper_2603_14859_b300 import api
    L = W.L
    w = W.weights.astype(np.float32)
    if ws is None:
        ws = api.alloc_workspace(W.J, x.shape[0], L, k, prec)
        ws.fill_(0xFF)                                 # stale workspace contents must not matter
    idx, dist = api.discrepancy_topk(y, x, L, w, k, prec, ws)
    st = api.topk_status(ws)
    assert st[0] == 0 and st[2] == 0, f"status {st}"
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    yn, xn = y.cpu().numpy()[:, :L], x.cpu().numpy()[:, :L].astype(np.float64)
    oi, od = orc.topk(yn, xn, w.astype(np.float64), k)
    swaps, worst = check_topk_sets(idx, oi, od, lambda vj, dn: orc.pair_dist(yn, xn, w, vj, dn), L, tau_extra)
    # returned distances: exact fp32 re-score of the returned draws
    J = W.J
    ref = orc.pair_dist(yn, xn, w, np.repeat(np.arange(J), k), idx.reshape(-1)).reshape(J, k)
    assert np.all(np.abs(dist - ref) <= 4 * L * 2.0**-24 * ref + 1e-30)
    # sorted ascending by (distance, index)
    assert np.all((np.diff(dist, axis=1) > 0) | ((np.diff(dist, axis=1) == 0) & (np.diff(idx, axis=1) > 0)))
    return swaps, worst, st[1]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_topk_brain_2tcm_small(orc, prec):
    W, y, x = _gpu_case("brain_fdg_2tcm", 300, 5000, orc)          # 3 voxel tiles (ragged), 40 draw tiles (ragged)
    swaps, worst, fallback = _compare(orc, W, y, x, 100, prec)
    assert swaps <= 3


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_topk_raclopride_two_models(orc, prec):
    W, y, x = _gpu_case("raclopride_lpntpet", 260, 3000, orc)     # 60 frames, FP32 K = 192 (3 K-blocks)
    _compare(orc, W, y, x, 50, prec)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_topk_totalbody_rev_irr(orc, prec):
    W, y, x = _gpu_case("totalbody_fdg", 129, 20000, orc)          # 29 frames, K = 128 (2 K-blocks)
    _compare(orc, W, y, x, 200, prec)


@pytest.mark.parametrize("prec", [0, 2])
def test_topk_many_compactions(orc, prec):
    """k small against a long draw stream: the candidate lists are compacted many times."""
    W, y, x = _gpu_case("brain_fdg_2tcm", 64, 60000, orc)
    _compare(orc, W, y, x, 5, prec)


@pytest.mark.parametrize("k", [1, 7])
def test_topk_tiny_and_k_edges(orc, k):
    W, y, x = _gpu_case("brain_fdg_2tcm", 5, 9, orc)               # N = 9 < one tile
    for prec in (0, 2):
        _compare(orc, W, y, x, k, prec)
        _compare(orc, W, y, x, 9, prec)                            # k = N


def test_noise_free_recovery():
    """A voxel whose TAC is exactly draw i*'s TAC gets i* first with distance 0."""
    from paper_2603_14859_b300 import api
    W = S.workload("brain_fdg_2tcm", J=4, N_per_model=4)
    lo, hi = S.PRIORS[S.TCM2_IRR]
    N = 7000
    th = api.sample_prior(3, S.TCM2_IRR, lo, hi, N)
    x = api.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, th)
    stars = [0, 4095, 6999, 1234, 5000]
    y = x[stars].clone()
    for prec in (0, 1, 2):
        idx, dist = api.discrepancy_topk(y, x, W.L, W.weights.astype(np.float32), 10, prec)
        assert idx[:, 0].cpu().tolist() == stars
        assert torch.all(dist[:, 0] == 0)


def test_ties_resolved_by_index():
    from paper_2603_14859_b300 import api
    W = S.workload("brain_fdg_2tcm", J=4, N_per_model=4)
    lo, hi = S.PRIORS[S.TCM2_IRR]
    th = api.sample_prior(3, S.TCM2_IRR, lo, hi, 500)
    x = api.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, th)
    x[300] = x[17]
    x[450] = x[17]
    y = x[17:18].clone()
    for prec in (0, 2):
        idx, dist = api.discrepancy_topk(y, x, W.L, W.weights.astype(np.float32), 3, prec)
        assert idx[0].cpu().tolist() == [17, 300, 450]


def test_many_ties_at_the_kth_distance():
    """Ties that fill the k-th distance's bin past the gather capacity (radix fallback)
    and a scan whose distances all tie (a single distinct value): the accepted set is
    the lowest indices, in every exact mode."""
    from paper_2603_14859_b300 import api
    W = S.workload("brain_fdg_2tcm", J=4, N_per_model=4)
    lo, hi = S.PRIORS[S.TCM2_IRR]
    th = api.sample_prior(5, S.TCM2_IRR, lo, hi, 600)
    x = api.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, th)
    x[300:500] = x[17]
    y = x[17:18].clone()
    w = W.weights.astype(np.float32)
    for prec in (0, 2):
        idx, dist = api.discrepancy_topk(y, x, W.L, w, 10, prec)
        assert idx[0].cpu().tolist() == [17] + list(range(300, 309))
        assert torch.all(dist[0] == 0)
    xe = x[:250].clone()
    xe[:] = x[40]
    for prec in (0, 1, 2):
        idx, dist = api.discrepancy_topk(y, xe, W.L, w, 10, prec)
        assert idx[0].cpu().tolist() == list(range(10))
        assert torch.all(dist[0] == dist[0, 0])


def test_argument_errors():
    from paper_2603_14859_b300 import api
    from paper_2603_14859_b300._lib import AbcError
    y = torch.zeros((4, 24), device="cuda")
    x = torch.zeros((10, 24), device="cuda")
    w = np.ones(22, np.float32)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(AbcError):
        api.discrepancy_topk(y, x, 22, w, 11, 0, workspace=ws)          # k > N
    with pytest.raises(AbcError):
        api.discrepancy_topk(y, x, 22, -w, 3, 0, workspace=ws)          # negative weights
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(AbcError) as e:
        api.discrepancy_topk(y, x, 22, w, 3, 0, workspace=ws)
    assert e.value.code == -3


@pytest.mark.parametrize("prec,k,mode", [(2, 10, 1), (1, 50, 1), (2, 10, 3), (1, 50, 5), (0, 2, 1)])
def test_uncertified_voxels_match_oracle(orc, prec, k, mode):
    """Voxels whose first net cannot be certified.  The FP32 form resolves them by the
    exact scan over the tiles whose segment-feature bound admits the net's k-th distance
    (with k = 2 many voxels of this case).  The split form queues them for its second
    tensor-core pass (rescue) with the threshold their net's k-th distance asks for.  The
    test hook abc_debug_force_rescue steers the path: mode 1 fails every first net, so
    every voxel of this 512-voxel scan is queued and the rescue resolves it; mode 3 fails
    the rescue nets too, so every voxel then takes the exact scan bounded by its first
    net's k-th distance; mode 5 limits the queue to a quarter of the voxels, so the rest
    take the exact scan at once.  The accepted sets still match the oracle's."""
    from paper_2603_14859_b300 import _lib, api
    W, y, x = _gpu_case("raclopride_lpntpet", 512, 20000, orc)
    L = W.L
    ws = api.alloc_workspace(W.J, x.shape[0], L, k, prec)
    ws.fill_(0xFF)                                     # stale workspace contents must not matter
    _lib.check(_lib.lib().abc_debug_force_rescue(mode))
    try:
        swaps, worst, scanned = _compare(orc, W, y, x, k, prec, ws=ws)
        st = api.topk_status(ws)
    finally:
        _lib.check(_lib.lib().abc_debug_force_rescue(0))
    if prec == 0:
        assert scanned > 0
    elif mode == 1:
        assert st[3] == W.J, f"status {st}"
    elif mode == 3:
        assert st[3] == W.J and st[1] == W.J, f"status {st}"
    else:
        assert st[3] == W.J // 4 and st[1] >= W.J - W.J // 4, f"status {st}"
    assert swaps == 0


@pytest.mark.parametrize("name,J,n,k,prec", [("raclopride_lpntpet", 700, 40000, 50, 2),
                                             ("raclopride_lpntpet", 700, 40000, 50, 1),
                                             ("brain_fdg_2tcm", 300, 5000, 100, 0),
                                             ("brain_fdg_2tcm", 5, 100, 7, 2)])
def test_kd_row_order_matches_oracle(orc, name, J, n, k, prec):
    """The k-d row order (tile-aligned splits of the voxels' and of each pilot group's
    draws) changes only which draw tiles a pass can skip: with the test hook
    abc_debug_order forcing it (mode 2) on scans far below its size threshold, the accepted
    sets match the oracle's and equal, index for index, those of the Morton order (mode 1).
    The cases: 6 ragged voxel tiles against 625 draw tiles in three pilot groups whose runs
    start off the tile grid; a single-group FP32 case; and a scan too small for the k-d
    order (100 draws), which keeps the Morton order."""
    from paper_2603_14859_b300 import _lib, api
    W, y, x = _gpu_case(name, J, n, orc)
    L, w = W.L, W.weights.astype(np.float32)
    out = {}
    try:
        for mode in (1, 2):
            _lib.check(_lib.lib().abc_debug_order(mode))
            ws = api.alloc_workspace(W.J, x.shape[0], L, k, prec)
            ws.fill_(0xFF)
            if mode == 2:
                swaps, worst, _ = _compare(orc, W, y, x, k, prec, ws=ws)
                assert swaps <= 3
            idx, dist = api.discrepancy_topk(y, x, L, w, k, prec, ws)
            st = api.topk_status(ws)
            assert st[0] == 0, f"status {st}"
            out[mode] = (idx.cpu().numpy(), dist.cpu().numpy())
    finally:
        _lib.check(_lib.lib().abc_debug_order(0))
    assert np.array_equal(out[1][0], out[2][0])
    assert np.array_equal(out[1][1], out[2][1])

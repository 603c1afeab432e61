"""Helpers shared by the GPU parity tests (comparison rules only, no method arithmetic)."""
import numpy as np

EPS32 = 2.0**-24


def check_topk_sets(gpu_idx, orc_idx, orc_dist, pair_dist_fn, L, tau_extra=0.0):
    """Accepted sets must match except for draws whose fp64 distance lies within the
    near-tie band tau * d_(k) of the oracle's k-th distance, tau = 16 L eps32 (+ tau_extra).
    Returns (n_voxels_with_swaps, max_band_swaps)."""
    J, k = orc_idx.shape
    tau = 16 * L * EPS32 + tau_extra
    swaps, worst = 0, 0
    for j in range(J):
        g, o = set(gpu_idx[j].tolist()), set(orc_idx[j].tolist())
        if g == o:
            continue
        diff = sorted(g ^ o)
        assert all(d >= 0 for d in diff), f"voxel {j}: invalid index in {diff}"
        dk = orc_dist[j, -1]
        dd = pair_dist_fn(np.full(len(diff), j), np.asarray(diff))
        bad = [n for n, d in zip(diff, dd) if abs(d - dk) > tau * max(dk, 1e-300)]
        assert not bad, f"voxel {j}: draws {bad[:5]} differ outside the tie band (d_k={dk})"
        swaps += 1
        worst = max(worst, len(diff))
    return swaps, worst

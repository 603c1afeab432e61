"""Bounded device waits of the fused tensor-core kernel.

Every barrier wait of the fused kernel gives up after a limit, flags
ABC_ERR_TIMEOUT, waits for the copies and MMAs its CTA still has in flight,
frees its tensor memory and returns.  The test-only hook abc_debug_inject_stall
makes the TMA producer skip one draw tile, so the waits behind that tile run
out after a shortened limit (nothing faults or spins without end).  The status
must say so, and the next ordinary call in the same process must return exactly
what it returned before the stall."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_14859_b300 import synth as S

pytestmark = pytest.mark.gpu


def _case(J=300, N=5000, seed=21):
    from paper_2603_14859_b300 import api
    W = S.workload("brain_fdg_2tcm", J=4, N_per_model=4)
    lo, hi = S.PRIORS[S.TCM2_IRR]
    th = api.sample_prior(seed, S.TCM2_IRR, lo, hi, N)
    x = api.simulate(S.TCM2_IRR, W.ts, W.te, W.inp, th)
    rng = np.random.default_rng(seed)
    pick = torch.from_numpy(rng.integers(0, N, J)).cuda()
    noise = torch.from_numpy(rng.standard_normal((J, x.shape[1]))).float().cuda()
    y = (x[pick] * (1 + 0.1 * noise)).contiguous()
    return y, x, W.L, W.weights.astype(np.float32)


@pytest.mark.parametrize("prec", [0, 1])
def test_stalled_producer_times_out_and_the_next_call_is_exact(prec):
    from paper_2603_14859_b300 import _lib, api
    y, x, L, w = _case()
    k = 50
    ws = api.alloc_workspace(y.shape[0], x.shape[0], L, k, prec)
    ref_idx, ref_dist = api.discrepancy_topk(y, x, L, w, k, prec, ws)
    assert api.topk_status(ws)[0] == _lib.ABC_OK
    lib = _lib.lib()
    _lib.check(lib.abc_debug_inject_stall(0, 50_000_000))        # withhold every CTA's first draw tile; 50 ms waits
    try:
        api.discrepancy_topk(y, x, L, w, k, prec, ws)
        st = api.topk_status(ws)
    finally:
        _lib.check(lib.abc_debug_inject_stall(-1, 0))
    assert st[0] == _lib.ABC_ERR_TIMEOUT
    torch.cuda.synchronize()
    # the context, its tensor memory and the workspace are usable again
    for _ in range(2):
        idx, dist = api.discrepancy_topk(y, x, L, w, k, prec, ws)
        assert api.topk_status(ws)[0] == _lib.ABC_OK
        assert torch.equal(idx, ref_idx) and torch.equal(dist, ref_dist)


def test_noalloc_variant_reports_its_timeout():
    from paper_2603_14859_b300 import _lib, api
    y, x, L, w = _case(J=200, N=4000, seed=22)
    k, prec = 20, 0
    ref_idx, ref_dist = api.discrepancy_topk(y, x, L, w, k, prec)
    lib = _lib.lib()
    P = ctypes.c_void_p
    s = P(torch.cuda.current_stream().cuda_stream)

    def call():
        idx = torch.full((y.shape[0], k), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((y.shape[0], k), -7.0, dtype=torch.float32, device="cuda")
        _lib.check(lib.abc_discrepancy_topk_noalloc(P(y.data_ptr()), y.shape[0], y.shape[1], P(x.data_ptr()),
                                                    x.shape[0], x.shape[1], L, w.ctypes.data_as(P), k, prec,
                                                    P(idx.data_ptr()), P(dist.data_ptr()), s))
        st = np.zeros(8, np.int32)
        _lib.check(lib.abc_topk_status_noalloc(st.ctypes.data_as(P), s))
        return idx, dist, st

    _lib.check(lib.abc_debug_inject_stall(0, 50_000_000))
    try:
        _, _, st = call()
    finally:
        _lib.check(lib.abc_debug_inject_stall(-1, 0))
    assert st[0] == _lib.ABC_ERR_TIMEOUT
    idx, dist, st = call()
    assert st[0] == _lib.ABC_OK
    assert torch.equal(idx, ref_idx) and torch.equal(dist, ref_dist)


def test_stall_hook_argument_checks():
    from paper_2603_14859_b300 import _lib
    lib = _lib.lib()
    assert lib.abc_debug_inject_stall(0, 10) == _lib.ABC_ERR_ARG           # below 1 ms
    assert lib.abc_debug_inject_stall(0, 20_000_000_000) == _lib.ABC_ERR_ARG
    _lib.check(lib.abc_debug_inject_stall(-1, 0))

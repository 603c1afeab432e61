"""The allocation-free discrepancy + top-k entry point.

It is for callers that may not allocate device memory (a host framework that
owns the device-memory budget, a pipeline that forbids allocation while
running, a plugin given only its inputs and outputs): its scratch is a fixed
64 MiB array inside the library.  Through the C ABI, two calls in a row must
return exactly what the workspace entry point returns for the same inputs, and
sizes beyond the fixed scratch must be refused.  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs(J, N, L, seed):
    from paper_2603_14859_b300 import api
    from paper_2603_14859_b300 import synth as S
    W = S.workload("brain_fdg_2tcm", J=4, N_per_model=4)
    lo, hi = S.PRIORS[S.TCM2_IRR]
    th = api.sample_prior(seed, S.TCM2_IRR, lo, hi, N)
    x = api.simulate(S.TCM2_IRR, W.ts[:L], W.te[:L], W.inp, th)
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, N, J)
    y = x[torch.from_numpy(pick).cuda()] * (1 + 0.1 * torch.from_numpy(rng.standard_normal((J, x.shape[1]))).float().cuda())
    return y.contiguous(), x, W.weights[:L].astype(np.float32)


def _noalloc(y, x, L, w, k, prec):
    from paper_2603_14859_b300._lib import check, lib
    J, N = y.shape[0], x.shape[0]
    idx = torch.full((J, k), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((J, k), -7.0, dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    check(lib().abc_discrepancy_topk_noalloc(ctypes.c_void_p(y.data_ptr()), J, y.shape[1],
                                             ctypes.c_void_p(x.data_ptr()), N, x.shape[1], L,
                                             w.ctypes.data_as(ctypes.c_void_p), k, prec,
                                             ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(dist.data_ptr()), s))
    return idx, dist


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_workspace_entry_point_twice(prec):
    from paper_2603_14859_b300 import api
    L, k = 22, 100
    for call, (J, N, seed) in enumerate([(300, 5000, 11), (257, 7001, 12)]):
        y, x, w = _inputs(J, N, L, seed)
        ref_idx, ref_dist = api.discrepancy_topk(y, x, L, w, k, prec)
        idx, dist = _noalloc(y, x, L, w, k, prec)
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_idx), f"call {call}: accepted draws differ"
        assert torch.equal(dist, ref_dist), f"call {call}: distances differ"


def test_noalloc_refuses_sizes_beyond_its_scratch():
    from paper_2603_14859_b300._lib import ABC_ERR_UNSUPPORTED, lib
    from paper_2603_14859_b300 import api
    J, N, L, k = 250_000, 100_000, 60, 500
    assert api.workspace_size(J, N, L, k, 1) > (64 << 20)
    w = np.ones(L, np.float32)
    P = ctypes.c_void_p
    fake = P(256)
    rc = lib().abc_discrepancy_topk_noalloc(fake, J, 64, fake, N, 64, L, w.ctypes.data_as(P), k, 1, fake, fake, None)
    assert rc == ABC_ERR_UNSUPPORTED
    assert b"64" in lib().abc_last_error() or b"scratch" in lib().abc_last_error()

"""The C-ABI library loads and exports every function include/*.h declares;
host-side argument validation and sizing work without a GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(abc_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2603_14859_b300.csrc import build
    build.build()
    from paper_2603_14859_b300 import _lib
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_2603_14859_b300 import _lib
    assert set(_lib.EXPORTS) == set(names)


def test_feng_input_host_only(lib):
    from paper_2603_14859_b300 import api
    c, a0, a1, a2 = api.feng_input([4e4, 1e4, 8e3], [1.0, 0.03, 0.01])
    assert c.tolist() == [1.0, 0.03, 0.01]
    assert a0.tolist() == [-1.8e4, 1e4, 8e3] and a1.tolist() == [4e4, 0.0, 0.0] and not a2.any()


def test_workspace_size_rules(lib):
    from paper_2603_14859_b300 import api
    a = api.workspace_size(1000, 50000, 22, 100, 0)
    b = api.workspace_size(1000, 50000, 22, 100, 1)
    assert a > 0 and b > 0
    assert a == api.workspace_size(1000, 50000, 22, 100, 0)
    assert api.workspace_size(2000, 50000, 22, 100, 0) > a
    for bad in [(0, 10, 5, 1, 0), (10, 5, 5, 6, 0), (10, 10, 62, 1, 0), (10, 10, 5, 1, 7), (10, 4096, 5, 2049, 0)]:
        assert lib.abc_workspace_size(*bad) == 0


def test_argument_validation_without_gpu(lib):
    """Invalid calls are rejected on the host before anything is enqueued."""
    from paper_2603_14859_b300 import _lib
    w = np.ones(22, np.float32)
    P = ctypes.c_void_p
    fake = P(256)
    rc = lib.abc_discrepancy_topk(fake, 10, 24, fake, 5, 24, 22, w.ctypes.data_as(P), 6, 0, fake, 1 << 20, fake,
                                  fake, None)
    assert rc == _lib.ABC_ERR_ARG and b"k" in lib.abc_last_error()
    rc = lib.abc_discrepancy_topk(fake, 10, 24, fake, 50, 22, 22, w.ctypes.data_as(P), 6, 0, fake, 1 << 20, fake,
                                  fake, None)
    assert rc == _lib.ABC_ERR_ARG                         # ldx not a multiple of 4
    lo = np.zeros(4)
    hi = np.ones(4)
    assert lib.abc_sample_prior(1, 0, lo.ctypes.data_as(P), hi.ctypes.data_as(P), 9, 10, 0, fake, 9, None) \
        == _lib.ABC_ERR_ARG                              # P > 8
    assert lib.abc_sample_prior(1, 0, hi.ctypes.data_as(P), lo.ctypes.data_as(P), 4, 10, 0, fake, 4, None) \
        == _lib.ABC_ERR_ARG                              # hi < lo
    off = np.array([0, 10], np.int64)
    assert lib.abc_model_select(fake, 3, 2, off.ctypes.data_as(P), 17, fake, fake, None) == _lib.ABC_ERR_ARG
    assert lib.abc_profile_events(fake, None) == _lib.ABC_ERR_ARG


def test_simulate_rejects_bad_schedules(lib):
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    ts = np.array([0.0, 2.0])
    te = np.array([3.0, 4.0])                  # overlapping frames
    c = np.array([1.0])
    z = np.zeros(1)
    fr = _lib.Frames(2, ts.ctypes.data, te.ctypes.data)
    pe = _lib.PolyExp(1, c.ctypes.data, c.ctypes.data, z.ctypes.data, z.ctypes.data)
    rc = lib.abc_simulate(0, ctypes.byref(fr), ctypes.byref(pe), P(256), 10, 4, P(256), 4, None)
    assert rc == _lib.ABC_ERR_ARG and b"overlap" in lib.abc_last_error()


def test_batch_and_tuning_validation_without_gpu(lib):
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    w = np.ones(22, np.float32)
    scans = (_lib.Scan * 2)()
    for i in range(2):
        scans[i] = _lib.Scan(256, 10, 24, 256, 50, 24, 22, w.ctypes.data, 5, 256, 256)
    assert lib.abc_batch_workspace_size(scans, 2, 1) > lib.abc_workspace_size(10, 50, 22, 5, 1)
    assert lib.abc_batch_workspace_size(scans, 0, 1) == 0
    assert lib.abc_batch_workspace_size(scans, 65, 1) == 0
    bad = _lib.Tuning(96, 2, 16, 1.5)
    rc = lib.abc_batch_discrepancy_topk(scans, 2, 1, ctypes.byref(bad), P(256), 1 << 30, None)
    assert rc == _lib.ABC_ERR_ARG and b"bn" in lib.abc_last_error()
    bad = _lib.Tuning(64, 2, 12, 1.5)
    assert lib.abc_set_default_tuning(ctypes.byref(bad)) == _lib.ABC_ERR_ARG
    t = _lib.Tuning()
    assert lib.abc_default_tuning(1, ctypes.byref(t)) == 0 and t.bn in (64, 128)
    scans[1].k = 51                                   # k > N in the second scan
    rc = lib.abc_batch_discrepancy_topk(scans, 2, 1, None, P(256), 1 << 30, None)
    assert rc == _lib.ABC_ERR_ARG


def test_learned_sizes_and_validation_without_gpu(lib):
    """Learned-proposal entry points: sizes and host-side argument checks (nothing enqueued)."""
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    assert lib.abc_mlp_param_count(30, 256, 8) == 256 * 30 + 256 + 256 * 256 + 256 + 8 * 256 + 8
    assert lib.abc_mlp_param_count(0, 256, 8) == 0
    assert lib.abc_mlp_workspace_size(30, 256, 8, 100) >= 4 * (100 * 256 * 4 + 100 * 8 * 2)
    assert lib.abc_mlp_workspace_size(30, 256, 8, 0) == 0
    assert lib.abc_mlp_init(1, 0, 256, 8, P(16), None) == _lib.ABC_ERR_ARG
    assert lib.abc_mlp_init(1, 30, 256, 8, None, None) == _lib.ABC_ERR_ARG
    assert lib.abc_mlp_forward(P(16), 30, 256, 8, P(16), 0, P(16), P(16), 1 << 30, None) == _lib.ABC_ERR_ARG
    assert lib.abc_mlp_forward(P(16), 30, 256, 8, P(16), 100, P(16), P(16), 16, None) == _lib.ABC_ERR_WORKSPACE
    assert lib.abc_mlp_loss_grad(P(16), 30, 256, 0, P(16), P(16), 10, P(16), 1 << 30, P(16), P(16),
                                 None) == _lib.ABC_ERR_ARG
    assert lib.abc_adam_update(P(16), P(16), P(16), P(16), 10, 1e-3, 1.0, 0.999, 1e-8, 1, None) == _lib.ABC_ERR_ARG
    assert lib.abc_adam_update(P(16), P(16), P(16), P(16), 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == _lib.ABC_ERR_ARG
    lo = np.array([0.0, 1.0]), np.array([1.0, 1.0])
    assert lib.abc_unit_box(P(16), 4, 8, 2, lo[0].ctypes.data, lo[1].ctypes.data, P(16), None) == _lib.ABC_ERR_ARG
    ts = np.array([0.0, 1.0]); te = np.array([1.0, 1.0])
    fr = _lib.Frames(2, ts.ctypes.data, te.ctypes.data)
    assert lib.abc_add_noise(P(16), 4, 4, ctypes.byref(fr), 109.8, 0.1, 0.1, 1, 0, P(16), 4,
                             None) == _lib.ABC_ERR_ARG       # empty frame
    assert "empty frame" in lib.abc_last_error().decode()
    w = np.ones(29, np.float32)
    lo4 = np.array([0.001, 0.001, 0.001, 0.03]); hi4 = np.array([1.0, 2.0, 0.5, 0.2])
    args = lambda k, M, T, amax: (P(16), 10, 32, 29, w.ctypes.data, P(16), P(16), T, amax, P(16),
                                  lo4.ctypes.data, hi4.ctypes.data, M, k, 1.0, 1, P(16), P(16), P(16), P(16), P(16),
                                  P(16), P(16), None, None, None)
    assert lib.abc_local_abc(*args(0, 100, 512, 2.5)) == _lib.ABC_ERR_ARG          # k = 0
    assert lib.abc_local_abc(*args(300, 1000, 512, 2.5)) == _lib.ABC_ERR_ARG       # k > 256
    assert lib.abc_local_abc(*args(100, 50, 512, 2.5)) == _lib.ABC_ERR_ARG         # M < k
    assert lib.abc_local_abc(*args(100, 1000, 512, 2.0)) == _lib.ABC_ERR_ARG       # k2 + k3 beyond the table
    assert lib.abc_local_abc(*args(100, 60000, 1024, 2.5)) == _lib.ABC_ERR_ARG     # shared memory
    assert "shared memory" in lib.abc_last_error().decode()
    assert lib.abc_local_abc_smem_bytes(512, 29, 10000) <= 227 * 1024
    assert lib.abc_local_abc_table(P(16), 512, 29, 28, P(16), None) == _lib.ABC_ERR_ARG   # ld < L
    assert lib.abc_local_abc_table(None, 512, 29, 29, P(16), None) == _lib.ABC_ERR_ARG


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_layout_of_mixed_widths_without_gpu(lib, prec):
    """A batch whose scans pack to different K widths is laid out at the widest: the
    host-side layout check passes (the call then stops at the workspace-size check),
    and the batch needs more than the sum of the narrower single-scan layouts (each
    scan alone as a one-scan batch: a single-scan call may give its split-form lists
    more room)."""
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    w = np.ones(61, np.float32)
    shapes = [(1000, 50000, 22, 50), (3000, 200000, 60, 100), (10, 5000, 29, 5), (1, 300, 61, 1)]
    scans = (_lib.Scan * len(shapes))()
    for i, (J, N, L, k) in enumerate(shapes):
        scans[i] = _lib.Scan(256, J, 64, 256, N, 64, L, w.ctypes.data, k, 256, 256)
    need = lib.abc_batch_workspace_size(scans, len(shapes), prec)
    alone = []
    for i in range(len(shapes)):
        one = (_lib.Scan * 1)(scans[i])
        alone.append(lib.abc_batch_workspace_size(one, 1, prec))
    if prec == 0:
        assert need > sum(alone) - 4 * 4096
    else:     # a scan alone may give its split-form lists more room than it gets in a batch
        assert need > max(alone)
    assert all(lib.abc_workspace_size(J, N, L, k, prec) == a for (J, N, L, k), a in zip(shapes, alone))
    rc = lib.abc_batch_discrepancy_topk(scans, len(shapes), prec, None, P(256), need - 256, None)
    assert rc == _lib.ABC_ERR_WORKSPACE
    assert b"workspace needs" in lib.abc_last_error()


def test_response_band_validation_without_gpu(lib):
    """abc_response_cri checks its arguments on the host before any launch."""
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    t = np.linspace(0, 60, 5).astype(np.float32)
    tp = t.ctypes.data_as(P)
    ok = dict(theta=P(16), ld=7, idx=P(16), J=10, k=50, first=0, last=100, t=tp, T=5)

    def call(**kw):
        a = dict(ok, **kw)
        return lib.abc_response_cri(a["theta"], a["ld"], a["idx"], a["J"], a["k"], a["first"], a["last"], a["t"],
                                    a["T"], P(16), P(16), P(16), None)
    assert call(ld=6) == _lib.ABC_ERR_ARG                 # fewer than the 7 lp-ntPET columns
    assert call(k=0) == _lib.ABC_ERR_ARG
    assert call(k=2049) == _lib.ABC_ERR_ARG
    assert call(J=-1) == _lib.ABC_ERR_ARG
    assert call(first=5, last=4) == _lib.ABC_ERR_ARG
    assert call(T=0) == _lib.ABC_ERR_ARG
    assert call(T=257) == _lib.ABC_ERR_ARG
    assert call(t=None) == _lib.ABC_ERR_ARG
    assert call(theta=None) == _lib.ABC_ERR_ARG
    nan = np.array([1.0, np.nan], np.float32)
    assert call(t=nan.ctypes.data_as(P), T=2) == _lib.ABC_ERR_ARG
    assert call(J=0) == _lib.ABC_OK                        # nothing to do, nothing launched


def test_l1_validation_without_gpu(lib):
    """abc_discrepancy_topk_l1 and its workspace size check their arguments on the host."""
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    w = np.ones(64, np.float32)
    wp = w.ctypes.data_as(P)
    assert lib.abc_l1_workspace_size(100, 0) == 0 and lib.abc_l1_workspace_size(-1, 5) == 0
    ws = lib.abc_l1_workspace_size(100, 50)
    assert ws >= 100 * (2 * 50 + 512) * 8

    def call(J=100, ldy=64, N=1000, ldx=64, L=60, w=wp, k=50, wsb=ws):
        return lib.abc_discrepancy_topk_l1(P(16), J, ldy, P(16), N, ldx, L, w, k, P(16), P(16), P(16), wsb, None)
    assert call(L=0) == _lib.ABC_ERR_ARG and call(L=65) == _lib.ABC_ERR_ARG
    assert call(k=0) == _lib.ABC_ERR_ARG and call(k=2049) == _lib.ABC_ERR_ARG
    assert call(N=49) == _lib.ABC_ERR_ARG                      # fewer draws than k
    assert call(ldy=59) == _lib.ABC_ERR_ARG and call(ldx=59) == _lib.ABC_ERR_ARG
    assert call(w=None) == _lib.ABC_ERR_ARG
    assert call(wsb=ws - 1) == _lib.ABC_ERR_ARG
    neg = np.ones(60, np.float32)
    neg[7] = -1.0
    assert call(w=neg.ctypes.data_as(P)) == _lib.ABC_ERR_ARG
    assert call(J=0, wsb=lib.abc_l1_workspace_size(0, 50)) == _lib.ABC_OK


def test_force_rescue_hook_mask_without_gpu(lib):
    """The second-pass test hook takes a mask of 1, 2 and 4; anything else is refused and
    leaves the hook as it was (off)."""
    from paper_2603_14859_b300 import _lib
    assert lib.abc_debug_force_rescue(8) == _lib.ABC_ERR_ARG
    assert b"mask" in lib.abc_last_error()
    assert lib.abc_debug_force_rescue(-1) == _lib.ABC_ERR_ARG
    assert lib.abc_debug_force_rescue(7) == _lib.ABC_OK
    assert lib.abc_debug_force_rescue(0) == _lib.ABC_OK


def test_order_hook_modes_without_gpu(lib):
    """The row-order test hook takes 0 (by scan size), 1 (Morton) or 2 (k-d); anything else
    is refused."""
    from paper_2603_14859_b300 import _lib
    assert lib.abc_debug_order(3) == _lib.ABC_ERR_ARG
    assert b"mode" in lib.abc_last_error()
    assert lib.abc_debug_order(-1) == _lib.ABC_ERR_ARG
    for m in (1, 2, 0):
        assert lib.abc_debug_order(m) == _lib.ABC_OK


def test_fallback_and_quantile_validation_without_gpu(lib):
    """Argument checks of the learned path's reliability calls, before any device work."""
    from paper_2603_14859_b300 import _lib
    P = ctypes.c_void_p
    assert lib.abc_fallback_scratch_size(0) == 0 and lib.abc_fallback_scratch_size(1) > 0
    assert lib.abc_quantile_scratch_size(0) == 0 and lib.abc_quantile_scratch_size(10) >= 40
    need = lib.abc_fallback_scratch_size(1000)
    assert lib.abc_fallback_rows(P(16), P(16), P(16), 0, 200, 0.0, P(16), P(16), P(16), need, None) == _lib.ABC_ERR_ARG
    assert lib.abc_fallback_rows(P(16), P(16), P(16), 1000, 0, 0.0, P(16), P(16), P(16), need, None) == _lib.ABC_ERR_ARG
    assert lib.abc_fallback_rows(P(16), None, None, 1000, 200, 0.1, P(16), P(16), P(16), need, None) \
        == _lib.ABC_ERR_ARG                                   # rel_max > 0 needs dmed and ynorm
    assert lib.abc_fallback_rows(P(16), P(16), P(16), 1000, 200, 0.0, P(16), P(16), P(16), need - 1, None) \
        == _lib.ABC_ERR_ARG
    assert b"scratch" in lib.abc_last_error()
    assert lib.abc_gather_rows(P(16), 4, P(16), P(16), 10, 5, P(16), 5, None) == _lib.ABC_ERR_ARG   # ld_src < width
    assert lib.abc_scatter_rows(None, 5, P(16), P(16), 10, 5, P(16), 5, None) == _lib.ABC_ERR_ARG
    w = np.ones(29, np.float32)
    qn = lib.abc_quantile_scratch_size(100)
    out = ctypes.c_float()
    for args in [(100, 9, 29, 29, 1.5), (100, 9, 65, 65, 0.5), (100, 0, 29, 29, 0.5), (100, 9, 29, 28, 0.5)]:
        J, k, L, ldy, q = args
        assert lib.abc_median_rel_quantile(P(16), J, k, P(16), ldy, L, w.ctypes.data, q, ctypes.byref(out), P(16),
                                           qn, None) == _lib.ABC_ERR_ARG, args

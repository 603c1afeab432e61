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

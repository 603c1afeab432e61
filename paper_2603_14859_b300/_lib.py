"""ctypes loader for libvpetabc.so (the C ABI in include/vpetabc.h).

The shared library is built in-tree by `paper_2603_14859_b300.csrc.build`.
There is no fallback: if the library is missing or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libvpetabc.so")

ABC_OK = 0
ABC_ERR_ARG = -1
ABC_ERR_CUDA = -2
ABC_ERR_WORKSPACE = -3
ABC_ERR_TIMEOUT = -4
ABC_ERR_UNSUPPORTED = -5
ABC_2TCM_IRR, ABC_2TCM_REV, ABC_MRTM, ABC_LPNTPET = 0, 1, 2, 3
ABC_FP32, ABC_BF16_RESCORE, ABC_SPLIT_DRAWS = 0, 1, 2

# every symbol the public header declares
EXPORTS = [
    "abc_feng_input", "abc_sample_prior", "abc_simulate", "abc_workspace_size", "abc_discrepancy_topk",
    "abc_topk_status", "abc_model_select", "abc_summarize", "abc_last_error", "abc_profile_events",
    "abc_debug_gemm_keys", "abc_discrepancy_topk_noalloc", "abc_default_tuning", "abc_set_default_tuning",
    "abc_batch_workspace_size", "abc_batch_discrepancy_topk", "abc_launch_info",
    "abc_mlp_param_count", "abc_mlp_workspace_size", "abc_mlp_init", "abc_mlp_features", "abc_mlp_forward",
    "abc_mlp_loss_grad", "abc_adam_update", "abc_add_noise", "abc_local_abc_smem_bytes", "abc_local_abc",
    "abc_unit_box", "abc_topk_work", "abc_local_abc_table", "abc_response_cri",
    "abc_l1_workspace_size", "abc_discrepancy_topk_l1", "abc_l1_status", "abc_topk_status_noalloc",
    "abc_debug_inject_stall", "abc_debug_force_rescue", "abc_debug_order", "abc_fallback_scratch_size", "abc_fallback_rows",
    "abc_gather_rows", "abc_scatter_rows", "abc_quantile_scratch_size", "abc_median_rel_quantile",
    "abc_mlp_status",
]


class Frames(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("t_start", ctypes.c_void_p), ("t_end", ctypes.c_void_p)]


class PolyExp(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int32), ("c", ctypes.c_void_p), ("a0", ctypes.c_void_p),
                ("a1", ctypes.c_void_p), ("a2", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("bn", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("pilot_stride", ctypes.c_int32),
                ("pilot_factor", ctypes.c_float)]


class Scan(ctypes.Structure):
    _fields_ = [("y_dev", ctypes.c_void_p), ("J", ctypes.c_int64), ("ldy", ctypes.c_int32), ("x_dev", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("ldx", ctypes.c_int32), ("L", ctypes.c_int32), ("w_host", ctypes.c_void_p),
                ("k", ctypes.c_int32), ("idx_dev", ctypes.c_void_p), ("dist_dev", ctypes.c_void_p)]


class AbcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError(f"{SO_PATH} is not built; run `python -m paper_2603_14859_b300.csrc.build`")
    L = ctypes.CDLL(SO_PATH)
    P, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    L.abc_feng_input.argtypes = [P, P, P, P, P, P]
    L.abc_sample_prior.argtypes = [u64, i32, P, P, i32, i64, i64, P, i32, P]
    L.abc_simulate.argtypes = [i32, ctypes.POINTER(Frames), ctypes.POINTER(PolyExp), P, i64, i32, P, i32, P]
    L.abc_workspace_size.argtypes = [i64, i64, i32, i32, i32]
    L.abc_workspace_size.restype = sz
    L.abc_discrepancy_topk.argtypes = [P, i64, i32, P, i64, i32, i32, P, i32, i32, P, sz, P, P, P]
    L.abc_topk_status.argtypes = [P, P, P]
    L.abc_model_select.argtypes = [P, i64, i32, P, i32, P, P, P]
    L.abc_summarize.argtypes = [P, i32, P, i32, P, P, P, P, i64, i32, P, i32, P, P, P, P, P]
    L.abc_last_error.restype = ctypes.c_char_p
    L.abc_profile_events.argtypes = [P, P]
    L.abc_discrepancy_topk_noalloc.argtypes = [P, i64, i32, P, i64, i32, i32, P, i32, i32, P, P, P]
    L.abc_topk_status_noalloc.argtypes = [P, P]
    L.abc_debug_inject_stall.argtypes = [i64, u64]
    L.abc_debug_force_rescue.argtypes = [i32]
    L.abc_debug_order.argtypes = [i32]
    L.abc_default_tuning.argtypes = [i32, ctypes.POINTER(Tuning)]
    L.abc_set_default_tuning.argtypes = [ctypes.POINTER(Tuning)]
    L.abc_launch_info.argtypes = [P, P, P]
    L.abc_batch_workspace_size.argtypes = [ctypes.POINTER(Scan), i32, i32]
    L.abc_batch_workspace_size.restype = sz
    L.abc_batch_discrepancy_topk.argtypes = [ctypes.POINTER(Scan), i32, i32, ctypes.POINTER(Tuning), P, sz, P]
    L.abc_debug_gemm_keys.argtypes = [P, i64, i32, P, i64, i32, i32, P, i32, P, sz, P, i64, P]
    f32 = ctypes.c_float
    f64 = ctypes.c_double
    L.abc_mlp_param_count.argtypes = [i32, i32, i32]
    L.abc_mlp_param_count.restype = sz
    L.abc_mlp_workspace_size.argtypes = [i32, i32, i32, i64]
    L.abc_mlp_workspace_size.restype = sz
    L.abc_mlp_init.argtypes = [u64, i32, i32, i32, P, P]
    L.abc_mlp_features.argtypes = [P, i64, i32, i32, P, P, P]
    L.abc_mlp_forward.argtypes = [P, i32, i32, i32, P, i64, P, P, sz, P]
    L.abc_mlp_loss_grad.argtypes = [P, i32, i32, i32, P, P, i64, P, sz, P, P, P]
    L.abc_adam_update.argtypes = [P, P, P, P, i64, f32, f32, f32, f32, i32, P]
    L.abc_add_noise.argtypes = [P, i64, i32, ctypes.POINTER(Frames), f64, f64, f64, u64, i64, P, i32, P]
    L.abc_unit_box.argtypes = [P, i64, i32, i32, P, P, P, P]
    L.abc_topk_work.argtypes = [P, P, P]
    L.abc_local_abc_smem_bytes.argtypes = [i32, i32, i32]
    L.abc_local_abc_table.argtypes = [P, i32, i32, i32, P, P]
    L.abc_local_abc_smem_bytes.restype = sz
    L.abc_response_cri.argtypes = [P, i32, P, i64, i32, i64, i64, P, i32, P, P, P, P]
    L.abc_l1_workspace_size.argtypes = [i64, i32]
    L.abc_l1_workspace_size.restype = sz
    L.abc_discrepancy_topk_l1.argtypes = [P, i64, i32, P, i64, i32, i32, P, i32, P, P, P, sz, P]
    L.abc_l1_status.argtypes = [P, i64, i32, P]
    L.abc_local_abc.argtypes = [P, i64, i32, i32, P, P, P, i32, f64, P, P, P, i32, i32, f32, u64,
                                P, P, P, P, P, P, P, P, P, P]
    L.abc_fallback_scratch_size.argtypes = [i64]
    L.abc_fallback_scratch_size.restype = sz
    L.abc_fallback_rows.argtypes = [P, P, P, i64, i32, f32, P, P, P, sz, P]
    L.abc_gather_rows.argtypes = [P, i32, P, P, i64, i32, P, i32, P]
    L.abc_scatter_rows.argtypes = [P, i32, P, P, i64, i32, P, i32, P]
    L.abc_quantile_scratch_size.argtypes = [i64]
    L.abc_quantile_scratch_size.restype = sz
    L.abc_median_rel_quantile.argtypes = [P, i64, i32, P, i32, i32, P, f64, P, P, sz, P]
    L.abc_mlp_status.argtypes = [P]
    for fn in ["abc_feng_input", "abc_sample_prior", "abc_simulate", "abc_discrepancy_topk", "abc_topk_status",
               "abc_model_select", "abc_summarize", "abc_debug_gemm_keys", "abc_profile_events",
               "abc_discrepancy_topk_noalloc", "abc_default_tuning", "abc_set_default_tuning",
               "abc_batch_discrepancy_topk", "abc_launch_info", "abc_mlp_init", "abc_mlp_features",
               "abc_mlp_forward", "abc_mlp_loss_grad", "abc_adam_update", "abc_add_noise", "abc_local_abc", "abc_unit_box", "abc_topk_work",
               "abc_local_abc_table", "abc_response_cri", "abc_discrepancy_topk_l1", "abc_l1_status",
               "abc_fallback_rows", "abc_gather_rows", "abc_scatter_rows", "abc_median_rel_quantile", "abc_mlp_status",
               "abc_topk_status_noalloc", "abc_debug_inject_stall", "abc_debug_force_rescue", "abc_debug_order"]:
        getattr(L, fn).restype = ctypes.c_int
    _lib = L
    return L


def check(rc: int):
    if rc != ABC_OK:
        raise AbcError(rc, lib().abc_last_error().decode())

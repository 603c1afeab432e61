"""Thin PyTorch-facing wrappers over the C ABI (argument marshalling only).

Device tensors are torch CUDA tensors; every call is enqueued on the current
torch CUDA stream unless `stream` is given.  All arithmetic runs in the CUDA
library; nothing here computes on the host beyond packing arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

PARAM_COUNT = {_lib.ABC_2TCM_IRR: 4, _lib.ABC_2TCM_REV: 5, _lib.ABC_MRTM: 3, _lib.ABC_LPNTPET: 7}


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def feng_input(beta, kappa):
    """Feng's three-exponential plasma input as poly-exponential arrays (c, a0, a1, a2)."""
    b = _np(beta, np.float64)
    k = _np(kappa, np.float64)
    outs = [np.zeros(3) for _ in range(4)]
    check(lib().abc_feng_input(*(o.ctypes.data_as(ctypes.c_void_p) for o in [b, k] + outs)))
    return outs


def sample_prior(seed, model, lo, hi, N, first_index=0, ldtheta=8, out=None, stream=None):
    lo = _np(lo, np.float64)
    hi = _np(hi, np.float64)
    P = len(lo)
    if out is None:
        out = torch.zeros((N, ldtheta), dtype=torch.float32, device="cuda")
    assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.shape[0] >= N
    check(lib().abc_sample_prior(seed, model, lo.ctypes.data_as(ctypes.c_void_p), hi.ctypes.data_as(ctypes.c_void_p),
                                 P, N, first_index, _ptr(out), out.shape[1], _stream(stream)))
    return out


class _HostArgs:
    """Keeps the host arrays of a frames / input struct alive for one call."""

    def __init__(self, ts, te, inp):
        self.ts = _np(ts, np.float64)
        self.te = _np(te, np.float64)
        self.arr = [_np(a, np.float64) for a in (inp.c, inp.a0, inp.a1, inp.a2)]
        self.frames = _lib.Frames(len(self.ts), self.ts.ctypes.data, self.te.ctypes.data)
        self.inp = _lib.PolyExp(len(self.arr[0]), *[a.ctypes.data for a in self.arr])


def simulate(model, ts, te, inp, theta, N=None, ldx=None, out=None, stream=None):
    """Frame-mean TACs for the first N rows of theta (N x ldtheta fp32, CUDA)."""
    N = theta.shape[0] if N is None else N
    L = len(ts)
    ldx = ldx or ((L + 3) // 4) * 4
    if out is None:
        out = torch.zeros((N, ldx), dtype=torch.float32, device="cuda")
    h = _HostArgs(ts, te, inp)
    check(lib().abc_simulate(model, ctypes.byref(h.frames), ctypes.byref(h.inp), _ptr(theta), N, theta.shape[1],
                             _ptr(out), out.shape[1], _stream(stream)))
    return out


def workspace_size(J, N, L, k, precision):
    n = lib().abc_workspace_size(J, N, L, k, precision)
    if n == 0:
        raise ValueError("abc_workspace_size: unsupported sizes")
    return n


def alloc_workspace(J, N, L, k, precision):
    n = workspace_size(J, N, L, k, precision)
    return torch.empty(n, dtype=torch.uint8, device="cuda")


def discrepancy_topk(y, x, L, w, k, precision=_lib.ABC_FP32, workspace=None, idx=None, dist=None, stream=None):
    """k nearest draws per voxel: returns (idx int32 J x k, dist fp32 J x k)."""
    J, N = y.shape[0], x.shape[0]
    w = _np(w, np.float32)
    if workspace is None:
        workspace = alloc_workspace(J, N, L, k, precision)
    if idx is None:
        idx = torch.empty((J, k), dtype=torch.int32, device="cuda")
    if dist is None:
        dist = torch.empty((J, k), dtype=torch.float32, device="cuda")
    check(lib().abc_discrepancy_topk(_ptr(y), J, y.shape[1], _ptr(x), N, x.shape[1], L,
                                     w.ctypes.data_as(ctypes.c_void_p), k, precision, _ptr(workspace),
                                     workspace.numel(), _ptr(idx), _ptr(dist), _stream(stream)))
    return idx, dist


def topk_status(workspace, stream=None):
    st = np.zeros(8, np.int32)
    check(lib().abc_topk_status(_ptr(workspace), st.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return tuple(int(v) for v in st)


def topk_work(workspace, stream=None):
    """(draw tiles processed, draw tiles without skipping) of the last main pass."""
    out = np.zeros(2, np.int64)
    check(lib().abc_topk_work(_ptr(workspace), out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return int(out[0]), int(out[1])


def debug_gemm_keys(y, x, L, w, precision, stream=None):
    """Raw tensor-core ranking keys d' = ||xh||^2 - 2 yh.xh for all pairs (test hook)."""
    J, N = y.shape[0], x.shape[0]
    w = _np(w, np.float32)
    ws = alloc_workspace(J, N, L, 1, precision)
    Jp, Np = -(-J // 128) * 128, -(-N // 128) * 128
    dump = torch.full((Jp, Np), float("nan"), dtype=torch.float32, device="cuda")
    check(lib().abc_debug_gemm_keys(_ptr(y), J, y.shape[1], _ptr(x), N, x.shape[1], L,
                                    w.ctypes.data_as(ctypes.c_void_p), precision, _ptr(ws), ws.numel(), _ptr(dump),
                                    Np, _stream(stream)))
    return dump[:J, :N], ws


def model_select(idx, offsets, prob=None, pref=None, stream=None):
    J, k = idx.shape
    off = _np(offsets, np.int64)
    M = len(off) - 1
    if prob is None:
        prob = torch.empty((J, M), dtype=torch.float32, device="cuda")
    if pref is None:
        pref = torch.empty(J, dtype=torch.int8, device="cuda")
    check(lib().abc_model_select(_ptr(idx), J, k, off.ctypes.data_as(ctypes.c_void_p), M, _ptr(prob), _ptr(pref),
                                 _stream(stream)))
    return prob, pref


def summarize(theta, offsets, nparams, has_ki, ki_cols, idx, pref=None, out=None, stream=None):
    """Posterior summaries -> (mean, sd, lo, hi), each J x (max(nparams) + 1) fp32."""
    J, k = idx.shape
    off = _np(offsets, np.int64)
    npar = _np(nparams, np.int32)
    hk = _np(has_ki, np.int32)
    kc = _np(ki_cols, np.int32)
    nc = int(npar.max()) + 1
    if out is None:
        out = [torch.empty((J, nc), dtype=torch.float32, device="cuda") for _ in range(4)]
    check(lib().abc_summarize(_ptr(theta), theta.shape[1], off.ctypes.data_as(ctypes.c_void_p), len(off) - 1,
                              npar.ctypes.data_as(ctypes.c_void_p), hk.ctypes.data_as(ctypes.c_void_p),
                              kc.ctypes.data_as(ctypes.c_void_p), _ptr(idx), J, k, _ptr(pref), nc,
                              *[_ptr(o) for o in out], _stream(stream)))
    return tuple(out)


def profile_events(start=None, stop=None):
    """Record torch.cuda.Event pair around the fused tensor-core kernel (None, None = off)."""
    a = ctypes.c_void_p(start.cuda_event) if start is not None else None
    b = ctypes.c_void_p(stop.cuda_event) if stop is not None else None
    check(lib().abc_profile_events(a, b))


def launch_info():
    """(grid, resident CTAs per SM) of the last fused-kernel launch, and the library's kernel-launch count."""
    g = ctypes.c_int64(0)
    r = ctypes.c_int32(0)
    n = ctypes.c_int64(0)
    check(lib().abc_launch_info(ctypes.byref(g), ctypes.byref(r), ctypes.byref(n)))
    return g.value, r.value, n.value


def l1_workspace_size(J, k):
    return int(lib().abc_l1_workspace_size(J, k))


def discrepancy_topk_l1(y, x, L, w, k, workspace=None, idx=None, dist=None, stream=None):
    """Per voxel the k nearest draws by the frame-weighted L1 distance -> (idx int32, dist fp32), J x k."""
    J, N = y.shape[0], x.shape[0]
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    if workspace is None:
        workspace = torch.empty(max(1, l1_workspace_size(J, k)), dtype=torch.uint8, device="cuda")
    if idx is None:
        idx = torch.empty((J, k), dtype=torch.int32, device="cuda")
    if dist is None:
        dist = torch.empty((J, k), dtype=torch.float32, device="cuda")
    check(lib().abc_discrepancy_topk_l1(_ptr(y), J, y.shape[1], _ptr(x), N, x.shape[1], L,
                                        w.ctypes.data_as(ctypes.c_void_p), k, _ptr(idx), _ptr(dist), _ptr(workspace),
                                        workspace.numel(), _stream(stream)))
    return idx, dist


def l1_status(workspace, J, k):
    v = ctypes.c_int32(0)
    check(lib().abc_l1_status(_ptr(workspace), J, k, ctypes.byref(v)))
    return v.value


def response_cri(theta, first, last, t, idx, out=None, stream=None):
    """Posterior mean and 95 % band of the lp-ntPET response function
    1 + (gamma / k2a) g(t) at the times t (minutes), over each voxel's accepted
    draws with global index in [first, last) -> (mean, lo, hi), each J x T fp32."""
    J, k = idx.shape
    tt = np.ascontiguousarray(np.asarray(t, dtype=np.float32).ravel())
    T = len(tt)
    if out is None:
        out = tuple(torch.empty((J, T), dtype=torch.float32, device="cuda") for _ in range(3))
    check(lib().abc_response_cri(_ptr(theta), theta.shape[1], _ptr(idx), J, k, int(first), int(last),
                                 tt.ctypes.data_as(ctypes.c_void_p), T, *[_ptr(o) for o in out], _stream(stream)))
    return out


def set_default_tuning(bn=None, ctas_per_sm=2, pilot_stride=16, pilot_factor=1.5):
    """Process-wide default tuning; bn=None restores the built-in per-precision defaults."""
    if bn is None:
        check(lib().abc_set_default_tuning(None))
        return
    t = _lib.Tuning(bn, ctas_per_sm, pilot_stride, pilot_factor)
    check(lib().abc_set_default_tuning(ctypes.byref(t)))


def default_tuning(precision=_lib.ABC_BF16_RESCORE):
    t = _lib.Tuning()
    check(lib().abc_default_tuning(precision, ctypes.byref(t)))
    return dict(bn=t.bn, ctas_per_sm=t.ctas_per_sm, pilot_stride=t.pilot_stride, pilot_factor=t.pilot_factor)


# ---------------------------------------------------------------- learned proposal + local ABC
def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def mlp_param_count(D, H, O):
    n = lib().abc_mlp_param_count(D, H, O)
    if n == 0:
        raise ValueError("abc_mlp_param_count: bad sizes")
    return n


def mlp_workspace_size(D, H, O, B):
    n = lib().abc_mlp_workspace_size(D, H, O, B)
    if n == 0:
        raise ValueError("abc_mlp_workspace_size: bad sizes")
    return n


def mlp_init(seed, D, H, O, out=None, stream=None):
    if out is None:
        out = torch.empty(mlp_param_count(D, H, O), dtype=torch.float32, device="cuda")
    check(lib().abc_mlp_init(seed, D, H, O, _ptr(out), _stream(stream)))
    return out


def mlp_features(y, L, w, out=None, stream=None):
    """Network inputs (J x (L+1)) of the voxel TACs y (J x ldy)."""
    J = y.shape[0]
    w = _np(w, np.float32)
    if out is None:
        out = torch.empty((J, L + 1), dtype=torch.float32, device="cuda")
    check(lib().abc_mlp_features(_ptr(y), J, y.shape[1], L, _vp(w), _ptr(out), _stream(stream)))
    return out


def mlp_forward(params, D, H, O, X, out=None, work=None, stream=None):
    B = X.shape[0]
    if out is None:
        out = torch.empty((B, O), dtype=torch.float32, device="cuda")
    if work is None:
        work = torch.empty(mlp_workspace_size(D, H, O, B), dtype=torch.uint8, device="cuda")
    check(lib().abc_mlp_forward(_ptr(params), D, H, O, _ptr(X), B, _ptr(out), _ptr(work), work.numel(),
                                _stream(stream)))
    return out


def mlp_loss_grad(params, D, H, P, X, T, grad=None, loss=None, work=None, stream=None):
    """(loss tensor [1], grad tensor) of the mean truncated-normal NLL."""
    B = X.shape[0]
    if grad is None:
        grad = torch.empty_like(params)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
    if work is None:
        work = torch.empty(mlp_workspace_size(D, H, 2 * P, B), dtype=torch.uint8, device="cuda")
    check(lib().abc_mlp_loss_grad(_ptr(params), D, H, P, _ptr(X), _ptr(T), B, _ptr(work), work.numel(), _ptr(grad),
                                  _ptr(loss), _stream(stream)))
    return loss, grad


def adam_update(params, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(lib().abc_adam_update(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), lr, beta1, beta2, eps,
                                t, _stream(stream)))


def unit_box(theta, N, P, lo, hi, out=None, stream=None):
    lo = _np(lo, np.float64)
    hi = _np(hi, np.float64)
    if out is None:
        out = torch.empty((N, P), dtype=torch.float32, device="cuda")
    check(lib().abc_unit_box(_ptr(theta), N, theta.shape[1], P, _vp(lo), _vp(hi), _ptr(out), _stream(stream)))
    return out


def add_noise(x, ts, te, half_life, q_lo, q_hi, seed, first_index=0, N=None, out=None, stream=None):
    N = x.shape[0] if N is None else N
    ts = _np(ts, np.float64)
    te = _np(te, np.float64)
    fr = _lib.Frames(len(ts), ts.ctypes.data, te.ctypes.data)
    if out is None:
        out = torch.empty_like(x)
    check(lib().abc_add_noise(_ptr(x), N, x.shape[1], ctypes.byref(fr), half_life, q_lo, q_hi, seed, first_index,
                              _ptr(out), out.shape[1], _stream(stream)))
    return out


def local_abc_smem_bytes(T, L, M):
    return lib().abc_local_abc_smem_bytes(T, L, M)


def local_abc_table(rows, stream=None):
    """The G table in the layout abc_local_abc reads: (T, L) rows -> (L, T) frame-major."""
    T, L = rows.shape
    out = torch.empty((L, T), device="cuda", dtype=torch.float32)
    check(lib().abc_local_abc_table(_ptr(rows), T, L, rows.stride(0), _ptr(out), _stream(stream)))
    return out


def local_abc(y, L, w, prop, table, a_max, cp_frames, lo, hi, M, k, seed, sigma_scale=1.0, dump=False, out=None,
              stream=None):
    """Importance-weighted local ABC (2TCM-irr) -> dict of device tensors; table is
    the frame-major (L, T) G table from local_abc_table."""
    J = y.shape[0]
    T = table.shape[1]
    w = _np(w, np.float32)
    lo = _np(lo, np.float64)
    hi = _np(hi, np.float64)
    dev = dict(device="cuda", dtype=torch.float32)
    if out is None:
        out = dict(mean=torch.empty((J, 5), **dev), sd=torch.empty((J, 5), **dev), lo=torch.empty((J, 5), **dev),
                   hi=torch.empty((J, 5), **dev), ess=torch.empty(J, **dev), dmed=torch.empty(J, **dev),
                   ynorm=torch.empty(J, **dev))
    if dump:
        out["u"] = torch.empty((J, M, 4), **dev)
        out["d"] = torch.empty((J, M), **dev)
    check(lib().abc_local_abc(_ptr(y), J, y.shape[1], L, _vp(w), _ptr(prop), _ptr(table), T, a_max, _ptr(cp_frames),
                              _vp(lo), _vp(hi), M, k, sigma_scale, seed, _ptr(out["mean"]), _ptr(out["sd"]), _ptr(out["lo"]),
                              _ptr(out["hi"]), _ptr(out["ess"]), _ptr(out["dmed"]), _ptr(out["ynorm"]),
                              _ptr(out.get("u")), _ptr(out.get("d")), _stream(stream)))
    return out


def fallback_rows(ess, dmed, ynorm, k, rel_max=None, stream=None):
    """Voxels the learned path hands to the global path: ESS below k/4 (or NaN), or (rel_max
    given) a median accepted distance above rel_max times sum_l w_l y_l^2.  Returns (rows, count):
    a device int32 tensor whose first count entries are those voxels, ascending, and the count
    as a one-element device tensor."""
    J = ess.shape[0]
    rows = torch.empty(J, dtype=torch.int32, device="cuda")
    count = torch.empty(1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(lib().abc_fallback_scratch_size(J), dtype=torch.uint8, device="cuda")
    check(lib().abc_fallback_rows(_ptr(ess), _ptr(dmed), _ptr(ynorm), J, k, float(rel_max or 0.0), _ptr(rows),
                                  _ptr(count), _ptr(scratch), scratch.numel(), _stream(stream)))
    return rows, count


def gather_rows(src, rows, count, n_rows, stream=None):
    """Device rows src[rows[i]] for i < count (count a device tensor; n_rows bounds it) -> (n_rows, width)."""
    out = torch.empty((n_rows, src.shape[1]), dtype=torch.float32, device="cuda")
    check(lib().abc_gather_rows(_ptr(src), src.stride(0), _ptr(rows), _ptr(count), n_rows, src.shape[1], _ptr(out),
                                out.stride(0), _stream(stream)))
    return out


def scatter_rows(src, rows, count, dst, stream=None):
    """dst[rows[i]] = src[i] for i < count (device count, at most src.shape[0]), in place."""
    check(lib().abc_scatter_rows(_ptr(src), src.stride(0), _ptr(rows), _ptr(count), src.shape[0], src.shape[1],
                                 _ptr(dst), dst.stride(0), _stream(stream)))
    return dst


def median_rel_quantile(dist, k, y, L, w, q, stream=None):
    """The q-quantile (numpy's linear interpolation) over voxels of the median accepted distance
    (column (k-1)/2 of dist) relative to sum_l w_l y_l^2."""
    J = dist.shape[0]
    w = _np(w, np.float32)
    scratch = torch.empty(lib().abc_quantile_scratch_size(J), dtype=torch.uint8, device="cuda")
    out = ctypes.c_float(0.0)
    check(lib().abc_median_rel_quantile(_ptr(dist), J, k, _ptr(y), y.stride(0), L, _vp(w), float(q), ctypes.byref(out),
                                        _ptr(scratch), scratch.numel(), _stream(stream)))
    return float(out.value)

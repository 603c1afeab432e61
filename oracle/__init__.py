"""FP64 CPU oracle for voxelwise ABC rejection — TEST INFRASTRUCTURE.

Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark use this package.  The CUDA library never imports, links or calls
it, and nothing here is shared with the CUDA sources.  See oracle.c for the
definitions each function restates and what pins it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               "-D_DEFAULT_SOURCE", _SRC, "-o", _SO + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_sample_prior.argtypes = [u64, ctypes.c_int, P, P, ctypes.c_int, i64, i64, P, ctypes.c_int]
        L.orc_simulate.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P, i64,
                                   ctypes.c_int, P, ctypes.c_int, ctypes.c_int]
        L.orc_tac_point.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, P, f64]
        L.orc_tac_point.restype = f64
        L.orc_Em.argtypes = [ctypes.c_int, f64, f64]
        L.orc_Em.restype = f64
        L.orc_gamma_variate.argtypes = [f64, f64, f64, f64]
        L.orc_gamma_variate.restype = f64
        L.orc_gl_nodes.argtypes = [P, P]
        L.orc_topk.argtypes = [P, i64, ctypes.c_int, P, i64, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P,
                               ctypes.c_int]
        L.orc_pair_dist.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P, P, i64, P]
        L.orc_model_select.argtypes = [P, i64, ctypes.c_int, P, ctypes.c_int, P, P]
        L.orc_summarize.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, P, P, P, i64, ctypes.c_int, P,
                                    ctypes.c_int, P, P, P, P]
        L.orc_topk_l1.argtypes = L.orc_topk.argtypes
        L.orc_response_cri.argtypes = [P, ctypes.c_int, P, i64, ctypes.c_int, i64, i64, P, ctypes.c_int, P, P, P]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_Phi.argtypes = [f64]
        L.orc_Phi.restype = f64
        L.orc_Phi_inv.argtypes = [f64]
        L.orc_Phi_inv.restype = f64
        L.orc_truncnorm01.argtypes = [f64, f64, f64]
        L.orc_truncnorm01.restype = f64
        L.orc_truncnorm01_logpdf.argtypes = [f64, f64, f64]
        L.orc_truncnorm01_logpdf.restype = f64
        L.orc_mlp_forward.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P]
        L.orc_mlp_loss_grad.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P]
        L.orc_mlp_loss_grad.restype = f64
        L.orc_local_abc.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int, P, P,
                                    ctypes.c_int, P, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def philox4x32_10(ctr, key):
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def sample_prior(seed, model, lo, hi, N, first=0, ldtheta=None):
    lo = _c(lo, np.float64)
    hi = _c(hi, np.float64)
    P = len(lo)
    ld = P if ldtheta is None else ldtheta
    th = np.zeros((N, ld), np.float32)
    lib().orc_sample_prior(seed, model, _p(lo), _p(hi), P, N, first, _p(th), ld)
    return th


def _pe(inp):
    return [_c(inp.c, np.float64), _c(inp.a0, np.float64), _c(inp.a1, np.float64), _c(inp.a2, np.float64)]


def simulate(model, ts, te, inp, theta, nthreads=0):
    """Frame-mean TACs (N x L, float64) for the rows of theta (float32)."""
    ts = _c(ts, np.float64)
    te = _c(te, np.float64)
    th = _c(theta, np.float32)
    N, ld = th.shape
    L = len(ts)
    pe = _pe(inp)
    x = np.zeros((N, L), np.float64)
    lib().orc_simulate(model, L, _p(ts), _p(te), len(pe[0]), *[_p(a) for a in pe], _p(th), N, ld, _p(x), L,
                       nthreads)
    return x


def tac_point(model, theta, inp, t):
    th = np.zeros(8, np.float32)
    th[: len(theta)] = theta
    pe = _pe(inp)
    return lib().orc_tac_point(model, _p(th), len(pe[0]), *[_p(a) for a in pe], float(t))


def Em(m, d, t):
    return lib().orc_Em(m, d, t)


def gamma_variate(t, tD, tP, alpha):
    return lib().orc_gamma_variate(t, tD, tP, alpha)


def gl_nodes():
    x = np.zeros(20)
    w = np.zeros(20)
    lib().orc_gl_nodes(_p(x), _p(w))
    return x, w


def topk(y, x, w, k, nthreads=0):
    """Per voxel the k nearest draws by (distance, index); returns (idx int32, dist float64)."""
    y = _c(y, np.float32)
    x = _c(x, np.float64)
    w = _c(w, np.float64)
    J, L = y.shape
    N = x.shape[0]
    idx = np.zeros((J, k), np.int32)
    dist = np.zeros((J, k), np.float64)
    rc = lib().orc_topk(_p(y), J, L, _p(x), N, x.shape[1], L, _p(w), k, _p(idx), _p(dist), nthreads)
    if rc != 0:
        raise ValueError("orc_topk failed")
    return idx, dist


def topk_l1(y, x, w, k, nthreads=0):
    """Per voxel the k nearest draws by the frame-weighted L1 distance, (distance, index) order."""
    y = _c(y, np.float32)
    x = _c(x, np.float64)
    w = _c(w, np.float64)
    J, L = y.shape
    N = x.shape[0]
    idx = np.zeros((J, k), np.int32)
    dist = np.zeros((J, k), np.float64)
    rc = lib().orc_topk_l1(_p(y), J, L, _p(x), N, x.shape[1], L, _p(w), k, _p(idx), _p(dist), nthreads)
    if rc != 0:
        raise ValueError("orc_topk_l1 failed")
    return idx, dist


def pair_dist(y, x, w, vj, dn):
    y = _c(y, np.float32)
    x = _c(x, np.float64)
    w = _c(w, np.float64)
    vj = _c(vj, np.int64)
    dn = _c(dn, np.int64)
    out = np.zeros(len(vj))
    lib().orc_pair_dist(_p(y), y.shape[1], _p(x), x.shape[1], y.shape[1], _p(w), _p(vj), _p(dn), len(vj), _p(out))
    return out


def model_select(idx, offsets):
    idx = _c(idx, np.int32)
    J, k = idx.shape
    off = _c(offsets, np.int64)
    M = len(off) - 1
    prob = np.zeros((J, M))
    pref = np.zeros(J, np.int8)
    if lib().orc_model_select(_p(idx), J, k, _p(off), M, _p(prob), _p(pref)) != 0:
        raise ValueError("index outside every model segment")
    return prob, pref


def summarize(theta, offsets, nparams, has_ki, ki_cols, idx, pref=None):
    """Posterior summaries; returns (mean, sd, lo, hi), each J x (Pmax + 1)."""
    th = _c(theta, np.float32)
    off = _c(offsets, np.int64)
    npar = _c(nparams, np.int32)
    hk = _c(has_ki, np.int32)
    kc = _c(ki_cols, np.int32)
    idx = _c(idx, np.int32)
    J, k = idx.shape
    Pmax = int(npar.max())
    outs = [np.zeros((J, Pmax + 1)) for _ in range(4)]
    pr = _c(pref, np.int8) if pref is not None else None
    lib().orc_summarize(_p(th), th.shape[1], _p(off), len(off) - 1, _p(npar), _p(hk), _p(kc), _p(idx), J, k,
                        _p(pr) if pr is not None else None, Pmax, *[_p(o) for o in outs])
    return tuple(outs)


def response_cri(theta, first, last, t, idx):
    """Posterior mean and 95 % band (type 7) of the lp-ntPET response function
    1 + (gamma / k2a) g(t) at the times t; each J x T."""
    th = _c(theta, np.float32)
    idx = _c(idx, np.int32)
    tt = _c(t, np.float64)
    J, k = idx.shape
    T = len(tt)
    outs = [np.zeros((J, T)) for _ in range(3)]
    lib().orc_response_cri(_p(th), th.shape[1], _p(idx), J, k, int(first), int(last), _p(tt), T,
                           *[_p(o) for o in outs])
    return tuple(outs)


def num_threads():
    return lib().orc_num_threads()


# ---------------------------------------------------------------- learned proposal (build extra)
def Phi(z):
    return lib().orc_Phi(float(z))


def Phi_inv(p):
    return lib().orc_Phi_inv(float(p))


def truncnorm01(mu, sigma, u):
    return lib().orc_truncnorm01(float(mu), float(sigma), float(u))


def truncnorm01_logpdf(mu, sigma, t):
    return lib().orc_truncnorm01_logpdf(float(mu), float(sigma), float(t))


def mlp_param_count(D, H, O):
    return H * D + H + H * H + H + O * H + O


def mlp_forward(params, D, H, O, X):
    prm = _c(params, np.float64)
    X = _c(X, np.float64)
    B = X.shape[0]
    out = np.zeros((B, O))
    z1 = np.zeros((B, H))
    z2 = np.zeros((B, H))
    lib().orc_mlp_forward(_p(prm), D, H, O, _p(X), B, _p(out), _p(z1), _p(z2))
    return out


def mlp_loss_grad(params, D, H, P, X, T):
    prm = _c(params, np.float64)
    X = _c(X, np.float64)
    T = _c(T, np.float64)
    g = np.zeros_like(prm)
    loss = lib().orc_mlp_loss_grad(_p(prm), D, H, P, _p(X), _p(T), X.shape[0], _p(g))
    return loss, g


def local_abc(u, mu, sigma, x, y, w, k, lo, hi, ki=True):
    """Importance-weighted local ABC for one voxel; returns dict of outputs."""
    u = _c(u, np.float64)
    M, P = u.shape
    x = _c(x, np.float64)
    y = _c(y, np.float32)
    w = _c(w, np.float64)
    mu = _c(mu, np.float64)
    sigma = _c(sigma, np.float64)
    lo = _c(lo, np.float64)
    hi = _c(hi, np.float64)
    nc = P + (1 if ki else 0)
    idx = np.zeros(k, np.int32)
    outs = [np.zeros(nc) for _ in range(4)]
    ess = np.zeros(1)
    lib().orc_local_abc(_p(u), _p(mu), _p(sigma), P, M, _p(x), x.shape[1], _p(y), _p(w), k, _p(lo), _p(hi),
                        1 if ki else 0, _p(idx), *[_p(o) for o in outs], _p(ess))
    return dict(idx=idx, mean=outs[0], sd=outs[1], lo=outs[2], hi=outs[3], ess=float(ess[0]))

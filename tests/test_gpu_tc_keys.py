"""Raw tensor-core ranking keys vs fp64: validates the tcgen05 / TMA / TMEM data
path of the discrepancy kernel (Alg. 1 step 4) before any top-k logic."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(J, N, L, seed=0):
    rng = np.random.default_rng(seed)
    base = np.abs(rng.normal(size=L)) * 1e4
    y = (base * (1 + 0.3 * rng.normal(size=(J, L)))).astype(np.float32)
    x = (base * (1 + 0.3 * rng.normal(size=(N, L)))).astype(np.float32)
    w = rng.uniform(0.1, 1.0, L).astype(np.float32)
    return y, x, w


def _pad(a):
    L = a.shape[1]
    ld = (L + 3) // 4 * 4
    out = np.zeros((a.shape[0], ld), np.float32)
    out[:, :L] = a
    return torch.from_numpy(out).cuda()


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("J,N,L", [(128, 128, 22), (200, 300, 22), (77, 1000, 60), (300, 129, 29)])
def test_gemm_keys_against_fp64(prec, J, N, L):
    from paper_2603_14859_b300 import api
    y, x, w = _case(J, N, L, seed=J + N)
    keys, ws = api.debug_gemm_keys(_pad(y), _pad(x), L, w, prec)
    torch.cuda.synchronize()
    keys = keys.cpu().numpy().astype(np.float64)
    mu = ws[256:256 + 4 * L].view(torch.float32).cpu().numpy().astype(np.float64)
    sw = np.sqrt(w.astype(np.float64))
    yh = sw * (y.astype(np.float64) - mu)
    xh = sw * (x.astype(np.float64) - mu)
    ynorm = (yh**2).sum(1)
    d_exact = ((yh[:, None, :] - xh[None, :, :]) ** 2).sum(-1)
    d_gpu = keys + ynorm[:, None]
    ry = np.sqrt(ynorm)[:, None]
    R = ry + np.sqrt(d_exact)
    if prec == 0:
        Kp = ((3 * L + 3 + 63) // 64) * 64
        cE = 3 * 2.0**-16 + (3 * Kp + L + 16) * 2.0**-24      # the kernel uses twice this
        bound = cE * (2 * ry * R + R * R)
        err = np.abs(d_gpu - d_exact)
        assert np.isfinite(keys).all()
        assert (err <= bound).all(), f"max err/bound = {(err / bound).max()}"
        return
    # split form (ABC_BF16_RESCORE and ABC_SPLIT_DRAWS): the voxel row rounded once, as the kernel
    # rounds it (fp32 centring and scaling, bf16 round to nearest); the draw row as bf16 hi + lo with
    # its residual folded into the norm column, so the key's error is at most
    # 2 sqrt(d) (||delta|| + 2^-16 R) plus the fp32 accumulation
    mu32 = mu.astype(np.float32)
    v32 = np.sqrt(w).astype(np.float32) * (y - mu32)
    yb = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float32).numpy()
    delta = yb.astype(np.float64) - v32
    c0 = -2.0 * (delta * v32).sum(1)[:, None]
    dn = np.sqrt((delta**2).sum(1))[:, None]
    Kp = ((2 * L + 3 + 63) // 64) * 64
    cacc = (3 * Kp + L + 16) * 2.0**-24
    err = np.abs(d_gpu - d_exact - c0)
    centring = 8 * 2.0**-24 * (ry * ry + R * R)        # fp32 vs fp64 centring and scaling of the rows
    bound = (2 * (dn + 2.0**-16 * R) * np.sqrt(d_exact) + 2.0**-15 * dn * (ry + R) + cacc * (2 * ry * R + R * R)
             + centring)
    assert np.isfinite(keys).all()
    assert (err <= bound).all(), f"max err/bound = {(err / bound).max()}"

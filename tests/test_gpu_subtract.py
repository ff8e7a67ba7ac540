"""GPU parity of the convolution and difference of image subtraction
(ipp_sub_apply; Sec. 2.2.4, Eqs. 8-10) with the oracle, on the same
coefficients.  The GPU evaluates the tile kernels and the 441-tap sums in FP32,
the oracle in FP64: |gpu - oracle| <= 1e-5 (|R| (x) |K|) + 1e-5 (|I| + |B|),
|K| the kernel's absolute value bounded by sum_n (sum_s |c_{n,s}|) |K_n| (every
spatial term is at most 1 in magnitude).  NaN exactly on the frame border the
kernel's support leaves."""
import numpy as np
import pytest
import torch
from scipy.signal import convolve2d

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _check(orc, gpu, I, R, coef, hw, sig, deg, sord, bord):
    o = orc.sub_apply(I, R, coef, hw=hw, sig=sig, deg=deg, sord=sord, bord=bord, tile=2 * hw + 1)
    g = host(gpu.sub_apply(dev(I), dev(R), coef, hw=hw, sig=sig, deg=deg, sord=sord, bord=bord))
    assert np.array_equal(np.isnan(g), np.isnan(o))
    B = orc.sub_basis(hw, sig, deg)
    nb, ns = B.shape[0], (sord + 1) * (sord + 2) // 2
    c = np.abs(np.asarray(coef[:nb * ns]).reshape(nb, ns)).sum(1)
    Kabs = np.tensordot(c, np.abs(B), 1)
    cabs = convolve2d(np.abs(R.astype(np.float64)), Kabs, mode="same")
    babs = np.abs(np.asarray(coef[nb * ns:])).sum() if bord >= 0 else 0.0
    tol = 1e-5 * cabs + 1e-5 * (np.abs(I) + babs)
    ok = ~np.isnan(o)
    assert np.all(np.abs(g[ok] - o[ok]) <= tol[ok])
    return int(ok.sum())


@pytest.mark.parametrize("hw,sig,deg,sord,bord", [(4, (1.0,), (2,), 0, -1), (6, (1.0, 2.5), (2, 0), 1, 1),
                                                  (10, (0.7, 1.5, 3.0), (6, 4, 2), 2, 1),
                                                  (12, (1.2, 3.0), (3, 1), 2, 2)])
def test_apply_parity(gpu, orc, hw, sig, deg, sord, bord):
    R, _ = synth.tiny_frame(517, 389, 81, n_stars=80, sky=300.0, flux=(3.0, 4.5))
    rng = np.random.default_rng(hw)
    I = (R + rng.normal(0, 5.0, R.shape)).astype(np.float32)
    nb = sum((d + 1) * (d + 2) // 2 for d in deg)
    ns = (sord + 1) * (sord + 2) // 2
    ng = (bord + 1) * (bord + 2) // 2 if bord >= 0 else 0
    coef = rng.normal(0, 0.05, nb * ns + ng)
    coef[0] = 0.9
    n = _check(orc, gpu, I, R, coef, hw, sig, deg, sord, bord)
    assert n == (517 - 2 * hw) * (389 - 2 * hw)


def test_apply_fitted_pair(gpu, orc):
    """coefficients fitted by the oracle on a synthetic pair, applied by both"""
    rng = np.random.default_rng(4)
    R, _ = synth.tiny_frame(400, 300, 82, n_stars=120, sky=200.0, flux=(3.5, 5.0))
    u = np.arange(-10, 11)
    G = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * 1.8 ** 2))
    I = (convolve2d(R.astype(np.float64), 0.9 * G / G.sum(), mode="same") + rng.normal(0, 3.0, R.shape) - 7.0)
    I = I.astype(np.float32)
    cx, cy = orc.sub_stamps(I, R, nsx=5, nsy=4, hw=10, fh=10, nsig=5.0)
    coef = orc.sub_fit(I, R, cx, cy, hw=10, fh=10, sord=1, bord=1)
    _check(orc, gpu, I, R, coef, 10, (0.7, 1.5, 3.0), (6, 4, 2), 1, 1)


def test_apply_views_and_errors(gpu, orc):
    R, _ = synth.tiny_frame(300, 200, 83, n_stars=30, sky=100.0)
    I = (R * 1.1).astype(np.float32)
    coef = np.zeros(7 + 1)
    coef[0], coef[7] = 1.0, 3.0
    sig, deg = (1.0, 2.5), (2, 0)
    o = orc.sub_apply(I, R, coef, hw=6, sig=sig, deg=deg, sord=0, bord=0, tile=13)
    out = torch.full((210, 320), -5.0, device="cuda")
    g = gpu.sub_apply(dev(I), dev(R), coef, hw=6, sig=sig, deg=deg, sord=0, bord=0, out=out[:200, :300])
    assert torch.all(out[:, 300:] == -5.0) and torch.all(out[200:] == -5.0)
    g = host(g)
    ok = ~np.isnan(o)
    assert np.array_equal(np.isnan(g), ~ok)
    assert np.max(np.abs(g[ok] - o[ok])) <= 1e-4 * np.max(np.abs(I))
    d = dev(I)
    with pytest.raises(gpu.IppError):
        gpu.sub_apply(d, dev(R), coef, hw=5, sig=sig, deg=deg, sord=0, bord=0)
    with pytest.raises(gpu.IppError):
        gpu.sub_apply(d, dev(R), coef, hw=6, sig=sig, deg=deg, sord=0, bord=0, out=d)
    with pytest.raises(gpu.IppError):
        gpu.sub_apply(d, dev(R), np.zeros(200), hw=6, sig=(1.0,) * 3, deg=(8, 8, 8), sord=0, bord=0)

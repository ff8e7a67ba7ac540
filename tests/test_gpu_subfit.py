"""GPU parity of the subtraction fit (ipp_sub_stamps, ipp_sub_normal,
ipp_sub_solve, ipp_sub_fit; Sec. 2.2.4, Eqs. 8-10) with the oracle.

Bars and why:
  stamps: exact -- the order statistics are selected on the values' bit
    patterns and the threshold is the same FP64 expression, so the candidate
    list must be identical;
  normal equations: both sides FP64, summed in different orders (the GPU
    convolves separably and sums per candidate first), so entries agree to
    1e-10 of their Cauchy-Schwarz scale sqrt(AtA_aa AtA_bb) (Atb: sqrt(AtA_aa
    sum I^2)) -- 44,100 footprint terms of unit round-off 1.1e-16;
  solution: compared in the metric of the normal matrix,
    sqrt((x - x0)' A (x - x0) / x0' A x0), the relative rms change of the
    fitted model over the footprints; on identical inputs the two FP64
    Cholesky solves agree to 1e-8 (the scaled matrix has condition ~1e11),
    end to end to 1e-6."""
import math

import numpy as np
import pytest
import torch
from scipy.signal import fftconvolve

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

SIG, DEG = (0.7, 1.5, 3.0), (6, 4, 2)


def _pair(R, sigma=1.6, ratio=0.9, sky=30.0, noise=3.0, seed=0):
    """I = R (x) K + sky + noise, K a normalised Gaussian (not in the basis' span)"""
    u = np.arange(-10, 11)
    G = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * sigma ** 2))
    K = ratio * G / G.sum()
    I = fftconvolve(R.astype(np.float64), K, mode="same") + sky
    I += np.random.default_rng(seed).normal(0, noise, R.shape)
    return I.astype(np.float32), R.astype(np.float32)


def _ragged():
    img, _ = synth.tiny_frame(517, 389, 41, n_stars=40, sky=300.0)
    return img


def _metric(A, x, x0):
    d = x - x0
    return math.sqrt(max(d @ A @ d, 0.0) / (x0 @ A @ x0))


def _stamps_both(gpu, orc, I, R, **kw):
    cx, cy, n = gpu.sub_stamps(dev(I), dev(R), **kw)
    n = int(host(n)[0])
    ocx, ocy = orc.sub_stamps(I, R, **kw)
    return host(cx)[:n], host(cy)[:n], ocx, ocy


@pytest.mark.parametrize("case", ["gradient_1k", "ragged", "nan_patches", "flat_region"])
def test_stamps_exact(gpu, orc, case):
    kw = dict(nsx=10, nsy=10, hw=10, fh=10, nsig=5.0)
    if case == "gradient_1k":
        R, _ = synth.frame_gradient_1k(1001)
    else:
        R = _ragged()
        kw = dict(nsx=4, nsy=3, hw=6, fh=6, nsig=5.0)
    I, R = _pair(R)
    if case == "nan_patches":
        # NaNs next to the brightest stars: their regions must fall back to the
        # next eligible pixel, or lose their candidate
        ocx, ocy = orc.sub_stamps(I, R, **kw)
        for k in range(0, len(ocx), 2):
            I[ocy[k] + 3, ocx[k] - 2] = np.nan
            R[ocy[k] - 9:ocy[k] - 7, ocx[k] + 4] = np.nan
        R[:, 100] = np.nan                      # a bad column
    if case == "flat_region":
        R[:150, :200] = 300.0                   # no star there: no candidate
        I[:150, :200] = 300.0
        R[200:260, 300:400] = np.nan            # an all-NaN block inside a region
    gcx, gcy, ocx, ocy = _stamps_both(gpu, orc, I, R, **kw)
    assert len(ocx) > 3
    assert np.array_equal(gcx, ocx) and np.array_equal(gcy, ocy)


def test_stamps_region_without_finite_pixels(gpu, orc):
    I, R = _pair(_ragged())
    R[:195, :259] = np.nan                      # region (0, 0) of 2 x 2 has no finite pixel
    gcx, gcy, ocx, ocy = _stamps_both(gpu, orc, I, R, nsx=2, nsy=2, hw=6, fh=6, nsig=5.0)
    assert np.array_equal(gcx, ocx) and np.array_equal(gcy, ocy)


def _normal_check(A, b, oA, ob, I_norm2):
    d = np.sqrt(np.diag(oA))
    assert np.all(np.abs(A - oA) <= 1e-10 * np.outer(d, d) + 1e-300)
    assert np.all(np.abs(b - ob) <= 1e-10 * d * math.sqrt(I_norm2) + 1e-300)


@pytest.mark.parametrize("orders", [(2, 1), (0, 0), (1, -1)])
def test_normal_parity(gpu, orc, orders):
    sord, bord = orders
    R, _ = synth.frame_gradient_1k(1001)
    I, R = _pair(R)
    cx, cy, n = gpu.sub_stamps(dev(I), dev(R))
    A, b = gpu.sub_normal(dev(I), dev(R), cx, cy, n, sord=sord, bord=bord)
    nn = int(host(n)[0])
    ocx, ocy = host(cx)[:nn], host(cy)[:nn]
    oA, ob = orc.sub_normal(I, R, ocx, ocy, sord=sord, bord=bord)
    fp = np.concatenate([I[y - 10:y + 11, x - 10:x + 11].ravel() for x, y in zip(ocx, ocy)]).astype(np.float64)
    _normal_check(host(A), host(b), oA, ob, float(fp @ fp))


def test_normal_small_basis_ragged(gpu, orc):
    """another basis, footprint and kernel size on a ragged frame"""
    I, R = _pair(_ragged())
    kw = dict(hw=6, fh=4, sig=(0.9, 2.2), deg=(3, 1), sord=1, bord=0)
    cx, cy, n = gpu.sub_stamps(dev(I), dev(R), nsx=4, nsy=3, hw=6, fh=4)
    A, b = gpu.sub_normal(dev(I), dev(R), cx, cy, n, **kw)
    nn = int(host(n)[0])
    ocx, ocy = host(cx)[:nn], host(cy)[:nn]
    oA, ob = orc.sub_normal(I, R, ocx, ocy, **kw)
    fp = np.concatenate([I[y - 4:y + 5, x - 4:x + 5].ravel() for x, y in zip(ocx, ocy)]).astype(np.float64)
    _normal_check(host(A), host(b), oA, ob, float(fp @ fp))


def test_solve_identical_inputs(gpu, orc):
    """the oracle's normal equations solved on both sides"""
    R, _ = synth.frame_gradient_1k(1001)
    I, R = _pair(R)
    ocx, ocy = orc.sub_stamps(I, R)
    oA, ob = orc.sub_normal(I, R, ocx, ocy)
    x0 = orc.chol_solve(oA, ob)
    A = torch.from_numpy(oA.copy()).cuda()
    b = torch.from_numpy(ob.copy()).cuda()
    c64, c32, st = gpu.sub_solve(A, b)
    assert int(host(st)[0]) == 0
    x = host(c64)
    assert _metric(oA, x, x0) < 1e-8
    assert np.array_equal(host(c32), x.astype(np.float32))


@pytest.mark.parametrize("which", ["gradient_1k", "survey_4k"])
def test_fit_end_to_end(gpu, orc, which):
    """ipp_sub_fit against the oracle's stamps, normal equations and solve; the
    4096^2 survey frame is the benchmark's workload"""
    if which == "gradient_1k":
        R, _ = synth.frame_gradient_1k(1001)
    else:
        R, _ = synth.frame_survey_4k()
    I, R = _pair(R, seed=3)
    o = gpu.sub_fit(dev(I), dev(R))
    assert int(host(o["status"])[0]) == 0
    n = int(host(o["n"])[0])
    ocx, ocy = orc.sub_stamps(I, R)
    assert np.array_equal(host(o["cx"])[:n], ocx) and np.array_equal(host(o["cy"])[:n], ocy)
    oA, ob = orc.sub_normal(I, R, ocx, ocy)
    x0 = orc.sub_fit(I, R, ocx, ocy)
    assert _metric(oA, host(o["coef64"]), x0) < 1e-6
    # the fitted kernel's sum is the flux ratio of the pair
    Kfit = np.tensordot(host(o["coef64"])[:49 * 6:6], orc.sub_basis(10), 1)
    assert abs(Kfit.sum() - 0.9) < 1e-2


def test_fit_without_candidates(gpu):
    """a frame with no star has no candidate: the normal matrix is zero and the
    solve reports status 1"""
    I = np.full((300, 300), 100.0, np.float32)
    R = I.copy()
    o = gpu.sub_fit(dev(I), dev(R), nsx=3, nsy=3)
    assert int(host(o["n"])[0]) == 0 and int(host(o["status"])[0]) == 1


def test_fit_rejects_bad_args(gpu):
    I = dev(np.zeros((64, 64), np.float32))
    with pytest.raises(Exception):
        gpu.sub_fit(I, I, sig=(0.7, -1.0, 3.0))
    with pytest.raises(Exception):
        gpu.sub_fit(I, I, sord=7)

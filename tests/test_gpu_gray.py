"""GPU parity of the gray-scale maps (Sec. 2.2.6) with the oracle.

Value-to-gray functions: the GPU computes in FP32, the oracle in FP64.  The
normalised value xn carries a relative error of a few 1e-7 (one rounding of
x - lo, of 1 / (hi - lo) and of the product); it reaches the gray value y
scaled by |dy / d ln xn|, which is 1 for linear, at most 1 for log, a for
power and ln(a) a / (a - 1) for exp (|ln a| / (1 - a) when a < 1).  The bar is
1e-6 times the larger of 1 and that factor.

Histogram equalisation: bin indices decide integers, and both sides form them
in FP32 with the same roundings, so the bin counts and the cumulative
distribution stored in the workspace are compared bit for bit with their
definition; the interpolated gray values (FP32 on the GPU, FP64 in the oracle)
agree to 1e-6."""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

KINDS = [("linear", 0, 1.0), ("log", 1, 1000.0), ("log", 1, 1e-3), ("power", 2, 0.5), ("power", 2, 3.0),
         ("exp", 3, 1000.0), ("exp", 3, 0.5), ("exp", 3, 1.001)]


def _cond(kind, a):
    if kind == 2:
        return a
    if kind == 3:
        return abs(math.log(a)) * (a / (a - 1.0) if a > 1.0 else 1.0 / (1.0 - a))
    return 1.0


def _planted(img, seed):
    """non-finite pixels at seeded positions"""
    img = img.copy()
    rng = np.random.default_rng(seed)
    H, W = img.shape
    for v in (np.nan, np.inf, -np.inf):
        img[rng.integers(0, H, 20), rng.integers(0, W, 20)] = v
    return img


def _hist_ref(img, nbins):
    """counts and cumulative distribution from the definition, in the FP32
    arithmetic the bin index is formed in"""
    f = img[np.isfinite(img)].astype(np.float32)
    mn, mx = f.min(), f.max()
    sc = np.float32(nbins) / np.float32(mx - mn)
    b = np.floor((f - mn) * sc).astype(np.int64)
    b = np.clip(b, 0, nbins - 1)
    cnt = np.bincount(b, minlength=nbins)
    cdf = (np.cumsum(cnt).astype(np.float64) / float(f.size)).astype(np.float32)
    return cnt.astype(np.uint32), cdf


def _ws_views(ws, nbins):
    raw = host(ws)
    nb = (nbins * 4 + 255) // 256 * 256
    cnt = raw[256:256 + nbins * 4].view(np.uint32)
    cdf = raw[256 + nb:256 + nb + nbins * 4].view(np.float32)
    return cnt, cdf


@pytest.mark.parametrize("name,kind,a", KINDS)
def test_gray_transform_parity(gpu, orc, name, kind, a):
    img, _ = synth.tiny_frame(1001, 389, 61, n_stars=60, sky=500.0, flux=(3.0, 5.0))
    img = _planted(img, 5)
    f = img[np.isfinite(img)]
    lo, hi = float(np.float32(np.percentile(f, 1))), float(np.float32(np.percentile(f, 99.5)))
    g = host(gpu.gray_transform(dev(img), kind, lo, hi, a=a))
    o = orc.gray_transform(img, kind, lo, hi, a=a)
    assert np.all(g[~np.isfinite(img)] == 0.0)
    assert np.max(np.abs(g - o)) <= 1e-6 * max(1.0, _cond(kind, a))
    assert g.min() >= 0.0 and g.max() <= 1.0 + 1e-6


def test_gray_transform_layouts(gpu, orc):
    """row pitch above the width, a base off the 16-byte boundary (scalar loads),
    ragged widths, one pixel"""
    base, _ = synth.tiny_frame(203, 77, 62, n_stars=10, sky=100.0)
    big = dev(base)
    for view in (big[:, :150], big[:, 1:], big[3:4, 5:6], big[:, :3]):
        ref = orc.gray_transform(host(view), 1, 80.0, 400.0, a=100.0)
        g = host(gpu.gray_transform(view, 1, 80.0, 400.0, a=100.0))
        assert np.max(np.abs(g - ref)) <= 1e-6
    out = torch.full((77, 256), -7.0, device="cuda")
    gpu.gray_transform(big, 0, 80.0, 400.0, out=out[:, :203])
    assert torch.all(out[:, 203:] == -7.0)
    assert np.max(np.abs(host(out[:, :203]) - orc.gray_transform(base, 0, 80.0, 400.0))) <= 1e-6


def test_gray_transform_errors(gpu):
    x = torch.zeros((8, 8), device="cuda")
    for kind, lo, hi, a in ((4, 0.0, 1.0, 1.0), (0, 1.0, 1.0, 1.0), (1, 0.0, 1.0, 0.0), (3, 0.0, 1.0, 1.0),
                            (2, 0.0, math.inf, 1.0)):
        with pytest.raises(gpu.IppError):
            gpu.gray_transform(x, kind, lo, hi, a=a)
    with pytest.raises(gpu.IppError):
        gpu.gray_transform(x, 0, 0.0, 1.0, out=x)


@pytest.mark.parametrize("which,nbins", [("gradient_1k", 4096), ("ragged", 2), ("ragged", 16384),
                                         ("lognormal", 1000)])
def test_hist_equalize_parity(gpu, orc, which, nbins):
    if which == "gradient_1k":
        img, _ = synth.frame_gradient_1k(1001)
    elif which == "ragged":
        img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0, flux=(3.0, 4.5))
        img = _planted(img, 6)
    else:
        rng = np.random.default_rng(9)
        img = np.exp(rng.normal(0.0, 1.5, (300, 1003))).astype(np.float32)
    out, ws = gpu.hist_equalize(dev(img), nbins=nbins)
    torch.cuda.synchronize()
    cnt, cdf = _ws_views(ws, nbins)
    rc, rf = _hist_ref(img, nbins)
    assert np.array_equal(cnt, rc)
    assert np.array_equal(cdf, rf)
    o = orc.hist_equalize(img, nbins=nbins)
    g = host(out)
    assert np.max(np.abs(g - o)) <= 1e-6
    assert np.all(g[~np.isfinite(img)] == 0.0)


def test_hist_equalize_edge_cases(gpu, orc):
    for img in (np.full((9, 13), 3.0, np.float32), np.full((4, 5), np.nan, np.float32),
                np.array([[np.nan, 2.0, np.inf]], np.float32), np.array([[7.0]], np.float32)):
        out, _ = gpu.hist_equalize(dev(img), nbins=64)
        assert not host(out).any()
        assert not orc.hist_equalize(img, nbins=64).any()
    img = np.array([[1.0, np.inf, 2.0, np.nan]], np.float32)
    g = host(gpu.hist_equalize(dev(img), nbins=16)[0])
    assert np.array_equal(g, orc.hist_equalize(img, nbins=16).astype(np.float32))
    # views: pitch above the width, unaligned base
    base, _ = synth.tiny_frame(203, 77, 63, n_stars=10, sky=100.0)
    big = dev(base)
    for view in (big[:, :150], big[:, 1:]):
        g = host(gpu.hist_equalize(view, nbins=256)[0])
        assert np.max(np.abs(g - orc.hist_equalize(host(view), nbins=256))) <= 1e-6
    x = torch.zeros((8, 8), device="cuda")
    with pytest.raises(ValueError):
        gpu.hist_equalize(x, nbins=1)
    with pytest.raises(gpu.IppError):
        gpu.hist_equalize(x, nbins=16, out=x)


def _big_frame():
    """8192^2 float32 (256 MiB, above L2): log-normal sky with a gradient and a
    block of NaN (a masked region)"""
    rng = np.random.default_rng(11)
    H = W = 8192
    img = rng.standard_normal((H, W), dtype=np.float32)
    img *= np.float32(0.4)
    np.exp(img, out=img)
    img *= np.float32(300.0)
    img += np.linspace(0.0, 200.0, W, dtype=np.float32)[None, :]
    img[4000:4100, 100:300] = np.nan
    return img


@pytest.mark.parametrize("which", ["survey_4k", "full_8k"])
def test_gray_full_size(gpu, orc, which):
    """the survey frame of the benchmark and the 8192^2 maximum case: equalise,
    then the log map, both compared on every pixel"""
    img = synth.frame_survey_4k()[0] if which == "survey_4k" else _big_frame()
    d = dev(img)
    out, ws = gpu.hist_equalize(d, nbins=4096)
    g = gpu.gray_transform(d, 1, 100.0, 2000.0, a=1000.0)
    torch.cuda.synchronize()
    cnt, cdf = _ws_views(ws, 4096)
    rc, rf = _hist_ref(img, 4096)
    assert np.array_equal(cnt, rc) and np.array_equal(cdf, rf)
    assert np.max(np.abs(host(out) - orc.hist_equalize(img, nbins=4096))) <= 1e-6
    assert np.max(np.abs(host(g) - orc.gray_transform(img, 1, 100.0, 2000.0, a=1000.0))) <= 1e-6

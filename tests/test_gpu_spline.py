"""GPU parity of the natural-spline background map (ipp_bg_subtract_spline,
the natural cubic spline reading of Sec. 2.2.2's interpolation back to full
resolution) against the oracle's FP64 map (orc_spline_map, pinned against
scipy's natural CubicSpline).

Tolerance: the GPU solves the nodes' tridiagonal systems and evaluates the
cubics in FP32; on node values of magnitude |B| the map and the subtracted
frame agree within 1e-5 max(|f|, |B|), like the Keys path."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _check(gpu, orc, img, mesh, **kw):
    H, W = img.shape
    ob, orr, _ = orc.bg_estimate(img, mesh=mesh, min_valid=1)
    B = orc.spline_map(ob, mesh, W, H)
    gsub, gb = gpu.bg_subtract_spline(dev(img), dev(ob), mesh=mesh, bkg_map=True, **kw)
    gsub, gb = host(gsub), host(gb)
    scale = np.maximum(np.abs(img), np.abs(B))
    assert np.all(np.abs(gb - B) <= 1e-5 * scale), np.max(np.abs(gb - B) / scale)
    assert np.all(np.abs(gsub - (img.astype(np.float64) - B)) <= 1e-5 * scale)
    return ob


@pytest.mark.parametrize("shape,mesh", [((389, 517), 32), ((1024, 1024), 64), ((221, 300), 24), ((40, 300), 64),
                                        ((300, 40), 64), ((70, 70), 32), ((33, 129), 16)])
def test_spline_parity(gpu, orc, shape, mesh):
    """ragged frames: partial last meshes, pixels beyond the outer nodes (the end
    lines), grids of one node row or column and of 2 x 2 nodes"""
    H, W = shape
    img, _ = synth.tiny_frame(W, H, 91, n_stars=6, sky=800.0) if H * W < 1 << 20 else synth.frame_gradient_1k(92)
    _check(gpu, orc, img, mesh)


def test_spline_curved_sky(gpu, orc):
    """a quadratic sky (the survey frame's shape, smaller): node second
    derivatives far from zero"""
    H, W = 640, 896
    yy, xx = np.mgrid[0:H, 0:W]
    sky = 1000 + 200 * (((xx - W / 2) / W) ** 2 + ((yy - H / 2) / H) ** 2)
    img = (sky + np.random.default_rng(4).normal(0, 5, (H, W))).astype(np.float32)
    _check(gpu, orc, img, 64)


def test_spline_u16_input(gpu, orc):
    """raw uint16 input with bias and flat fused into the read"""
    if not hasattr(torch, "uint16"):
        pytest.skip("torch without uint16")
    raw, flat, _ = synth.raw_calibrated_4k(5301, W=517, H=389, n_stars=30)
    f = orc.calibrate(raw, flat, bias=500.0)
    ob, _, _ = orc.bg_estimate(f, mesh=32)
    B = orc.spline_map(ob, 32, 517, 389)
    inv = dev((1.0 / flat.astype(np.float64)).astype(np.float32))
    traw = torch.from_numpy(raw.view(np.int16)).cuda().view(torch.uint16)
    gsub = host(gpu.bg_subtract_spline(traw, dev(ob), mesh=32, calib=(inv, 500.0)))
    scale = np.maximum(np.abs(f), np.abs(B))
    assert np.all(np.abs(gsub - (f.astype(np.float64) - B)) <= 2e-5 * scale)


def test_spline_survey_frame_full_size(gpu, orc):
    """the 4096^2 survey frame (mesh 128), the configuration the benchmark times"""
    img, _ = synth.frame_survey_4k()
    ob, _, _ = orc.bg_estimate(img, mesh=128)
    B = orc.spline_map(ob, 128, 4096, 4096)
    gsub, gb = gpu.bg_subtract_spline(dev(img), dev(ob), mesh=128, bkg_map=True)
    gb = host(gb)
    scale = np.maximum(np.abs(img), np.abs(B))
    assert np.all(np.abs(gb - B) <= 1e-5 * scale)

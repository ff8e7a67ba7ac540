"""GPU parity of the background steps (Sec. 2.2.2) against the FP64 oracle:
mesh statistics + filter (ipp_bg_estimate) and interpolation + subtraction
(ipp_bg_subtract), element by element on seeded frames.

Tolerances: mesh values 1e-5 relative (the statistics are exact order
statistics and double-float sums; only the final FP32 rounding and the
FP32-vs-FP64 median filter of even windows remain).  Subtracted pixels:
|d| <= 1e-5 * max(|f|, |B|) -- the Keys interpolation is evaluated in FP32
(relative rounding ~1e-7 of the background)."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host, rel_close

pytestmark = pytest.mark.gpu


def _cmp_mesh(gb, gr, ob, orr, rtol=1e-5, atol=1e-6):
    assert gb.shape == ob.shape
    okb = rel_close(gb, ob, rtol, atol)
    okr = rel_close(gr, orr, rtol, atol)
    assert okb.all(), f"bkg mismatch at {np.argwhere(~okb)[:5]}: {gb[~okb][:5]} vs {ob[~okb][:5]}"
    assert okr.all(), f"rms mismatch at {np.argwhere(~okr)[:5]}: {gr[~okr][:5]} vs {orr[~okr][:5]}"


@pytest.mark.parametrize("shape,mesh,seed", [((1024, 1024), 64, 1001), ((221, 300), 32, 7),
                                             ((130, 97), 16, 8), ((64, 64), 64, 9)])
def test_bg_estimate_parity(gpu, orc, shape, mesh, seed):
    H, W = shape
    if (H, W) == (1024, 1024):
        img, _ = synth.frame_gradient_1k(seed)
    else:
        img, _ = synth.tiny_frame(W, H, seed, n_stars=6)
    ob, orr, st = orc.bg_estimate(img, mesh=mesh)
    gb, gr, rb, rr, status = gpu.bg_estimate(dev(img), mesh=mesh, raw=True)
    torch.cuda.synchronize()
    assert int(host(status)[0]) == 0
    # raw (unfiltered) statistics, valid meshes
    v = st["valid"] == 1
    assert np.array_equal(host(rr) >= 0, v)
    _cmp_mesh(host(rb)[v], host(rr)[v], st["raw_bkg"][v], st["raw_rms"][v])
    _cmp_mesh(host(gb), host(gr), ob, orr)


def test_bg_estimate_survey_frame_full_size(gpu, orc):
    """4096^2 survey field with hot pixels and cosmic rays, 128 px meshes, the
    launch configuration of the benchmark: every mesh value against the oracle."""
    img, _ = synth.frame_survey_4k()
    ob, orr, st = orc.bg_estimate(img, mesh=128)
    gb, gr = gpu.bg_estimate(dev(img), mesh=128)
    _cmp_mesh(host(gb), host(gr), ob, orr)


@pytest.mark.parametrize("est", [0, 1, 2, 3])
def test_bg_estimators(gpu, orc, est):
    img, _ = synth.tiny_frame(256, 192, 21, n_stars=8)
    kw = dict(mesh=32, estimator=est, median_factor=3.0, mean_factor=2.0)
    ob, orr, _ = orc.bg_estimate(img, **kw)
    gb, gr = gpu.bg_estimate(dev(img), **kw)
    _cmp_mesh(host(gb), host(gr), ob, orr)


def test_bg_mask_and_invalid_fill(gpu, orc):
    img, _ = synth.tiny_frame(256, 256, 31, n_stars=5)
    mask = np.zeros(img.shape, np.uint8)
    mask[0:64, 0:64] = 1            # two fully masked meshes -> invalid, filled
    mask[100:140, 200:256] = 1      # partial masking
    img[70, 70] = np.nan            # non-finite pixel excluded
    ob, orr, st = orc.bg_estimate(img, mask=mask, mesh=32)
    assert (st["valid"] == 0).sum() >= 2
    gb, gr = gpu.bg_estimate(dev(img), mask=dev(mask), mesh=32)
    _cmp_mesh(host(gb), host(gr), ob, orr)


def test_bg_maxiters_and_filter_sizes(gpu, orc):
    img, _ = synth.tiny_frame(320, 256, 41, n_stars=12)
    for kw in (dict(mesh=32, maxiters=1), dict(mesh=32, maxiters=2, filter_size=1),
               dict(mesh=40, filter_size=5), dict(mesh=32, nsigma=2.0)):
        ob, orr, _ = orc.bg_estimate(img, **kw)
        gb, gr = gpu.bg_estimate(dev(img), **kw)
        _cmp_mesh(host(gb), host(gr), ob, orr)


def test_constant_frame_zero_residual(gpu):
    img = np.full((300, 260), 1234.5625, np.float32)
    t = dev(img)
    gb, gr = gpu.bg_estimate(t, mesh=64)
    sub = gpu.bg_subtract(t, gb, mesh=64)
    assert np.all(host(gb) == np.float32(1234.5625)) and np.all(host(gr) == 0)
    assert np.all(host(sub) == 0.0)


def test_no_valid_mesh_status(gpu):
    img = np.full((64, 64), np.nan, np.float32)
    gb, gr, rb, rr, status = gpu.bg_estimate(dev(img), mesh=32, raw=True)
    assert int(host(status)[0]) == 4   # IPP_ERR_NO_VALID_MESH
    assert np.all(host(gb) == 0)


@pytest.mark.parametrize("shape,mesh", [((1024, 1024), 64), ((221, 300), 32), ((77, 131), 8), ((40, 40), 64)])
def test_bg_subtract_parity(gpu, orc, shape, mesh):
    H, W = shape
    img, _ = synth.tiny_frame(W, H, 51, n_stars=5) if H < 1024 else synth.frame_gradient_1k(52)
    ob, orr, _ = orc.bg_estimate(img, mesh=mesh, min_valid=1)
    osub, obmap = orc.bg_subtract(img, ob, mesh)
    gsub, gbmap = gpu.bg_subtract(dev(img), dev(ob), mesh=mesh, bkg_map=True)
    gsub, gbmap = host(gsub), host(gbmap)
    scale = np.maximum(np.abs(img), np.abs(obmap))
    assert np.all(np.abs(gbmap - obmap) <= 1e-5 * scale)
    assert np.all(np.abs(gsub - osub) <= 1e-5 * scale)


def test_bg_subtract_pitched_input(gpu, orc):
    """row pitch larger than W (a view into a wider buffer)."""
    img, _ = synth.tiny_frame(203, 150, 61, n_stars=4)
    wide = np.zeros((150, 256), np.float32)
    wide[:, :203] = img
    tw = dev(wide)[:, :203]
    ob, orr, _ = orc.bg_estimate(img, mesh=32)
    gb, gr = gpu.bg_estimate(tw, mesh=32)
    _cmp_mesh(host(gb), host(gr), ob, orr)
    gsub = host(gpu.bg_subtract(tw, dev(ob), mesh=32))
    osub, obmap = orc.bg_subtract(img, ob, 32)
    assert np.all(np.abs(gsub - osub) <= 1e-5 * np.maximum(np.abs(img), np.abs(obmap)))


def test_uint16_calibrated_input(gpu, orc):
    """bias/flat correction fused into the first read: (raw - bias) * (1/flat)."""
    rng = np.random.default_rng(71)
    H, W = 200, 260
    raw = rng.integers(600, 3000, (H, W)).astype(np.uint16)
    flat = rng.uniform(0.9, 1.1, (H, W)).astype(np.float32)
    f = orc.calibrate(raw, flat, bias=500.0)
    ob, orr, _ = orc.bg_estimate(f, mesh=32)
    inv = dev((1.0 / flat.astype(np.float64)).astype(np.float32))
    traw = torch.from_numpy(raw.view(np.int16)).cuda().view(torch.uint16) if hasattr(torch, "uint16") else None
    if traw is None:
        pytest.skip("torch without uint16")
    gb, gr = gpu.bg_estimate(traw, mesh=32, calib=(inv, 500.0))
    # reciprocal-multiply vs divide differ in the last bit of each pixel: the
    # mesh statistics of such values agree to ~1e-7 relative
    _cmp_mesh(host(gb), host(gr), ob, orr, rtol=2e-5)


def _shaped_frame(kind, H=384, W=512, seed=0):
    """Meshes whose value distributions exercise every branch of the clip: a
    Gaussian sky, quantised (integer Poisson) values whose median bin holds
    thousands of equal values, bimodal mixtures whose median and bounds move
    into the core during the clip, heavy (Cauchy) tails, and one-sided
    exponential skew."""
    rng = np.random.default_rng(seed)
    if kind == "gauss":
        return rng.normal(1000, 30, (H, W)).astype(np.float32)
    if kind == "poisson":
        return rng.poisson(3.0, (H, W)).astype(np.float32)
    if kind == "poisson_big":
        return rng.poisson(40.0, (H, W)).astype(np.float32)
    if kind == "bimodal":
        m = rng.random((H, W)) < 0.15
        return np.where(m, rng.normal(1060, 10, (H, W)), rng.normal(1000, 10, (H, W))).astype(np.float32)
    if kind == "bimodal_wide":
        m = rng.random((H, W)) < 0.35
        return np.where(m, rng.normal(1300, 20, (H, W)), rng.normal(1000, 20, (H, W))).astype(np.float32)
    if kind == "cauchy":
        return (1000 + 5 * rng.standard_cauchy((H, W))).astype(np.float32)
    if kind == "expo":
        return (500 + rng.exponential(40, (H, W))).astype(np.float32)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["gauss", "poisson", "poisson_big", "bimodal", "bimodal_wide", "cauchy", "expo"])
@pytest.mark.parametrize("mesh", [128, 64])
def test_bg_estimate_distribution_shapes(gpu, orc, kind, mesh):
    img = _shaped_frame(kind, seed=sum(map(ord, kind)))
    ob, orr, st = orc.bg_estimate(img, mesh=mesh)
    gb, gr, rb, rr, status = gpu.bg_estimate(dev(img), mesh=mesh, raw=True)
    v = st["valid"] == 1
    _cmp_mesh(host(rb)[v], host(rr)[v], st["raw_bkg"][v], st["raw_rms"][v])
    _cmp_mesh(host(gb), host(gr), ob, orr)


@pytest.mark.parametrize("scale", [1e-20, 1e-6, 1e12])
def test_bg_estimate_extreme_scales(gpu, orc, scale):
    """Histogram windows far from unit scale: tiny values take the FP64
    branch of the clip statistics, large ones the double-float branch."""
    img, _ = synth.tiny_frame(256, 192, 91, n_stars=6)
    img = (img.astype(np.float64) * scale).astype(np.float32)
    ob, orr, st = orc.bg_estimate(img, mesh=64)
    gb, gr, rb, rr, status = gpu.bg_estimate(dev(img), mesh=64, raw=True)
    v = st["valid"] == 1
    assert v.all()
    _cmp_mesh(host(rb)[v], host(rr)[v], st["raw_bkg"][v], st["raw_rms"][v], atol=1e-30)
    _cmp_mesh(host(gb), host(gr), ob, orr, atol=1e-30)


def _timed_bg(gpu, t, **kw):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    out = gpu.bg_estimate(t, raw=True, **kw)
    e.record()
    torch.cuda.synchronize()
    return out, s.elapsed_time(e)


def test_fill_large_grid_bounded_time(gpu, orc):
    """Grids of 128 x 128 and 64 x 64 meshes (the two-pass fill path): all
    meshes masked returns IPP_ERR_NO_VALID_MESH at once; a single valid mesh in
    a corner (every other node filled from a ring far away) and a masked block
    match the oracle's fill and filter.  Each call is bounded in time (the fill
    is computed once per node, not once per window element)."""
    img = np.random.default_rng(3).normal(100.0, 5.0, (512, 512)).astype(np.float32)
    t = dev(img)
    mask = np.ones(img.shape, np.uint8)
    (gb, gr, rb, rr, st), ms = _timed_bg(gpu, t, mask=dev(mask), mesh=4, min_valid=4)
    assert int(host(st)[0]) == 4 and np.all(host(gb) == 0) and ms < 50.0, ms
    mask[:8, :8] = 0  # one valid mesh, top-left, of a 64 x 64 grid (the oracle's fill is cubic in k)
    (gb, gr, rb, rr, st), ms = _timed_bg(gpu, t, mask=dev(mask), mesh=8, min_valid=4)
    ob, orr, _ = orc.bg_estimate(img, mask=mask, mesh=8, min_valid=4)
    assert int(host(st)[0]) == 0 and ms < 200.0, ms
    _cmp_mesh(host(gb), host(gr), ob, orr)
    mask[:] = 0
    mask[100:400, 60:300] = 1
    (gb, gr, rb, rr, st), ms = _timed_bg(gpu, t, mask=dev(mask), mesh=8, min_valid=4)
    ob, orr, _ = orc.bg_estimate(img, mask=mask, mesh=8, min_valid=4)
    assert int(host(st)[0]) == 0 and ms < 200.0, ms
    _cmp_mesh(host(gb), host(gr), ob, orr)

"""The fused per-frame path (ipp_extract) against the oracle's whole path, on
the 1024^2 gradient field (mesh 64) and ragged frames: meshes and the
subtracted frame element-wise, then every source of the catalog matched one
to one (see catalog_match: components away from pixels within rounding of
the threshold are identical, and every matched source is compared on all of
its outputs)."""
import numpy as np
import pytest
import torch

import synth
from catalog_match import assert_catalog
from gpu_util import dev, float_ulp, host

pytestmark = pytest.mark.gpu

_OUT_KEYS = ("mesh_bkg", "mesh_rms", "sub", "labels", "x", "y", "cen_flags", "flux", "sky", "area", "n_ann",
             "phot_flags")


def host_catalog(out, stats=None):
    g = {k: host(out[k]) for k in _OUT_KEYS}
    g["n_src"] = int(host(out["n_src"])[0])
    st = {k: host(v) for k, v in (stats if stats is not None else out["stats"]).items()}
    return g, st


@pytest.mark.parametrize("which", ["gradient_1k", "ragged", "ragged_small_mesh"])
def test_extract_parity(gpu, orc, which):
    if which == "gradient_1k":
        img, _ = synth.frame_gradient_1k(1001)
        mesh = 64
    elif which == "ragged":
        img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0, flux=(3.0, 4.5))
        mesh = 32
    else:
        img, _ = synth.tiny_frame(777, 640, 78, n_stars=90, sky=800.0, flux=(2.8, 4.8))
        mesh = 24
    oc = orc.catalog(img, mesh=mesh)
    out = gpu.extract(dev(img), mesh=mesh)
    torch.cuda.synchronize()
    g, st = host_catalog(out)
    s = assert_catalog(orc, img, oc, g, st, mesh)
    assert s["matched"] >= 0.97 * s["oK"], s


@pytest.mark.parametrize("which", ["gradient_1k", "ragged"])
def test_extract_spline_parity(gpu, orc, which):
    """the catalog path with the natural-spline reading (interp = spline): the
    fused pass takes the background and the threshold's rms from the node tables
    of the filtered grids; the oracle composes its spline map with the same
    threshold, labeling, centroid and aperture"""
    if which == "gradient_1k":
        img, _ = synth.frame_gradient_1k(1001)
        mesh = 64
    else:
        img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0, flux=(3.0, 4.5))
        mesh = 32
    oc = orc.catalog(img, mesh=mesh, interp="spline")
    out = gpu.extract(dev(img), mesh=mesh, interp="spline")
    torch.cuda.synchronize()
    g, st = host_catalog(out)
    s = assert_catalog(orc, img, oc, g, st, mesh)
    assert s["matched"] >= 0.97 * s["oK"], s
    # the spline map differs from the Keys map, so the two catalogs' frames differ
    ok = gpu.extract(dev(img), mesh=mesh)
    assert not np.array_equal(host(ok["sub"]), g["sub"])


def test_extract_spline_u16(gpu, orc):
    """the spline reading on a raw uint16 frame with bias and flat fused into the read"""
    if not hasattr(torch, "uint16"):
        pytest.skip("torch without uint16")
    raw, flat, _ = synth.raw_calibrated_4k(5301, W=517, H=389, n_stars=30)
    f = orc.calibrate(raw, flat, bias=500.0)
    oc = orc.catalog(f, mesh=32, interp="spline")
    inv = dev((1.0 / flat.astype(np.float64)).astype(np.float32))
    traw = torch.from_numpy(raw.view(np.int16)).cuda().view(torch.uint16)
    out = gpu.extract(traw, calib=(inv, 500.0), mesh=32, interp="spline")
    torch.cuda.synchronize()
    g, st = host_catalog(out)
    s = assert_catalog(orc, f, oc, g, st, 32)
    assert s["matched"] >= 0.97 * s["oK"], s


def test_extract_repeatable(gpu):
    """two runs over the same frame give identical outputs, bit for bit: the
    component sums are integers (fixed point), so the order of the atomic
    merges does not matter."""
    img, _ = synth.frame_gradient_1k(1003)
    ex = gpu.Extractor(1024, 1024, gpu.BgConfig(mesh=64))
    t = dev(img)
    a = {k: host(v).copy() for k, v in ex(t).items()}
    sa = {k: host(v).copy() for k, v in ex.stats.items()}
    b = {k: host(v).copy() for k, v in ex(t).items()}
    sb = {k: host(v).copy() for k, v in ex.stats.items()}
    K = int(a["n_src"][0])
    for k in ("mesh_bkg", "mesh_rms", "sub", "labels", "n_src"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("x", "y", "flux", "sky", "area", "n_ann", "cen_flags", "phot_flags"):
        assert np.array_equal(a[k][:K], b[k][:K]), k
    for k in sa:
        assert np.array_equal(sa[k][:K], sb[k][:K]), k


def _raw_u16(seed, W=1024, H=768, n_stars=400, with_bias_map=False):
    """raw uint16 frame (bias 500, radial flat 0.9-1.1) at test size; optionally
    a per-pixel bias map (a column pattern of +-3 ADU around 500)"""
    raw, flat, _ = synth.raw_calibrated_4k(seed, W=W, H=H, n_stars=n_stars)
    bm = None
    if with_bias_map:
        j = np.arange(W, dtype=np.float64)
        bm = np.broadcast_to(500.0 + 3.0 * np.sin(j / 7.0), (H, W)).astype(np.float32).copy()
    return raw, flat, bm


def _u16_tensor(raw):
    if not hasattr(torch, "uint16"):
        pytest.skip("torch without uint16")
    return torch.from_numpy(raw.view(np.int16)).cuda().view(torch.uint16)


@pytest.mark.parametrize("with_bias_map", [False, True])
def test_extract_u16_parity(gpu, orc, with_bias_map):
    """raw uint16 input with bias (scalar or map) and flat fused into every read
    of ipp_extract, against the oracle's calibration (FP64 divide) followed by
    its whole path: the same matched-catalog comparison as the float frames."""
    raw, flat, bm = _raw_u16(5101 + with_bias_map, with_bias_map=with_bias_map)
    f = orc.calibrate(raw, flat, bias=500.0, bias_map=bm)
    mesh = 64
    oc = orc.catalog(f, mesh=mesh)
    inv = dev((1.0 / flat.astype(np.float64)).astype(np.float32))
    calib = (inv, 500.0) if bm is None else (inv, 500.0, dev(bm))
    out = gpu.extract(_u16_tensor(raw), mesh=mesh, calib=calib)
    torch.cuda.synchronize()
    g, st = host_catalog(out)
    s = assert_catalog(orc, f, oc, g, st, mesh)
    assert s["matched"] >= 0.97 * s["oK"], s


@pytest.mark.parametrize("with_bias_map", [False, True])
def test_bg_subtract_u16_parity(gpu, orc, with_bias_map):
    """ipp_bg_subtract on raw uint16 input: the calibrated frame minus the
    interpolated background, against the oracle on its calibrated frame."""
    raw, flat, bm = _raw_u16(5201 + with_bias_map, W=517, H=389, n_stars=60, with_bias_map=with_bias_map)
    f = orc.calibrate(raw, flat, bias=500.0, bias_map=bm)
    ob, orr, _ = orc.bg_estimate(f, mesh=32)
    osub, obmap = orc.bg_subtract(f, ob, 32)
    inv = dev((1.0 / flat.astype(np.float64)).astype(np.float32))
    calib = (inv, 500.0) if bm is None else (inv, 500.0, dev(bm))
    traw = _u16_tensor(raw)
    gb, gr = gpu.bg_estimate(traw, mesh=32, calib=calib)
    assert np.all(np.abs(host(gb) - ob) <= 2e-5 * np.abs(ob) + 1e-6)
    assert np.all(np.abs(host(gr) - orr) <= 2e-5 * np.abs(orr) + 1e-6)
    gsub = host(gpu.bg_subtract(traw, dev(ob), mesh=32, calib=calib))
    scale = np.maximum(np.abs(f), np.abs(obmap))
    assert np.all(np.abs(gsub - osub) <= 2e-5 * scale)

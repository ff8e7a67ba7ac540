"""GPU parity of detection on the smoothed frame (detection filter = 1) with the
oracle, from the GPU's own subtracted frame and mesh rms.  The smoothed value is
summed in FP32 on the GPU and FP64 in the oracle, so the masks may differ only
at pixels whose smoothed value lies within rounding (2e-5 relative) of
k rms(x, y); components touching no such pixel must match exactly."""
import numpy as np
import pytest
from scipy import ndimage

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

K3 = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], np.float64)


def _smoothed(sub):
    num = ndimage.convolve(sub.astype(np.float64), K3, mode="constant", cval=0.0)
    den = ndimage.convolve(np.ones_like(sub, np.float64), K3, mode="constant", cval=0.0)
    return num / den


@pytest.mark.parametrize("which", ["gradient_1k", "ragged"])
def test_filtered_detection_parity(gpu, orc, which):
    if which == "gradient_1k":
        img, _ = synth.frame_gradient_1k(1001)
        mesh = 64
    else:
        img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0, flux=(3.0, 4.5))
        mesh = 32
    H, W = img.shape
    g0 = gpu.extract(dev(img), mesh=mesh)
    g1 = gpu.extract(dev(img), mesh=mesh, filter=1)
    sub, rms = host(g1["sub"]), host(g1["mesh_rms"])
    assert np.array_equal(sub, host(g0["sub"]))  # the filter changes detection only
    om = orc.threshold(sub, rms, mesh, k=1.5, filtered=True)
    ol, oK, _ = orc.label(om, sub, min_area=5)
    gl, gK = host(g1["labels"]), int(host(g1["n_src"])[0])
    thr = 1.5 * orc.interp_map(rms, mesh, W, H)
    near = np.abs(_smoothed(sub) - thr) <= 2e-5 * np.maximum(np.abs(thr), 1.0)
    bad = np.unique(ol[near & (ol > 0)])
    ok = ~np.isin(ol, bad) & (ol > 0)
    pairs = np.unique(np.stack([ol[ok], gl[ok]], 1), axis=0)
    assert len(np.unique(pairs[:, 0])) == len(pairs) and len(np.unique(pairs[:, 1])) == len(pairs)
    assert np.all(gl[ok] > 0)
    if near.sum() == 0:
        assert gK == oK and np.array_equal(gl, ol)
    # smoothing removes most single-pixel noise islands: fewer candidates than unsmoothed
    assert gK < int(host(g0["n_src"])[0])

"""GPU parity of zscale (Sec. 2.2.6) with the oracle.  The samples and their
order are integer work: the counts (samples, good samples) must be equal.  The
fit is FP64 on both sides with sums in different orders, so the limits agree to
1e-9 relative; on the exactly solvable ramp-plus-outlier case (integer sums,
exact in any order) they are equal."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _both(gpu, orc, img, dimg=None, **kw):
    z, cnt = gpu.zscale(dev(img) if dimg is None else dimg, **kw)
    o1, o2, oc = orc.zscale(img, **kw)
    return host(z), tuple(int(v) for v in host(cnt)), (o1, o2), oc


@pytest.mark.parametrize("contrast,z", [(0.25, (0.0, 2503.5)), (1.0, (1.5, 1000.5))])
def test_closed_form(gpu, orc, contrast, z):
    img = np.full((20, 100), np.nan, np.float32)
    f = img.ravel()
    f[0:2000:2] = np.arange(1000, dtype=np.float32)
    f[1998] = 1e6
    g, gc, _, _ = _both(gpu, orc, img, contrast=contrast)
    assert tuple(g) == z and gc == (1000, 994)


@pytest.mark.parametrize("which", ["survey_4k", "gradient_1k", "ragged_nan", "sky_stars"])
def test_zscale_parity(gpu, orc, which):
    if which == "survey_4k":
        img = synth.frame_survey_4k()[0]
    elif which == "gradient_1k":
        img = synth.frame_gradient_1k(1001)[0]
    elif which == "ragged_nan":
        img, _ = synth.tiny_frame(517, 389, 71, n_stars=60, sky=400.0, flux=(3.0, 4.5))
        img = img.copy()
        img[50:60, :] = np.nan
    else:
        rng = np.random.default_rng(5)
        img = rng.normal(500.0, 20.0, (512, 512)).astype(np.float32)
        stars = rng.random(img.shape) < 0.03
        img[stars] = rng.uniform(1e4, 1e5, stars.sum()).astype(np.float32)
    for kw in (dict(), dict(n_samples=4096, contrast=0.5, krej=3.0, max_iter=8), dict(n_samples=37)):
        g, gc, o, oc = _both(gpu, orc, img, **kw)
        assert gc == oc
        assert np.allclose(g, o, rtol=1e-9, atol=0.0)


def test_zscale_views_and_edges(gpu, orc):
    img, _ = synth.tiny_frame(203, 77, 73, n_stars=10, sky=100.0)
    big = dev(img)
    for view in (big[:, 1:150], big[3:40, :]):
        g, gc, o, oc = _both(gpu, orc, host(view), dimg=view)
        assert gc == oc and np.allclose(g, o, rtol=1e-9, atol=0.0)
    # fewer than five samples, one pixel, nothing finite
    g, gc, o, oc = _both(gpu, orc, np.array([[3.0, np.nan, 1.0, 7.0]], np.float32))
    assert tuple(g) == (1.0, 7.0) and gc == (3, 3)
    g, gc, _, _ = _both(gpu, orc, np.array([[2.5]], np.float32))
    assert tuple(g) == (2.5, 2.5) and gc == (1, 1)
    z, cnt = gpu.zscale(dev(np.full((3, 3), np.nan, np.float32)))
    assert np.all(np.isnan(host(z))) and tuple(host(cnt)) == (0, 0)
    x = torch.zeros((8, 8), device="cuda")
    for bad in (dict(n_samples=0), dict(n_samples=4097), dict(contrast=0.0), dict(max_iter=-1)):
        with pytest.raises(gpu.IppError):
            gpu.zscale(x, **bad)

"""Pins of the oracle's zscale display limits (Sec. 2.2.6 names SAOimage's
zscale; the reading follows the published IRAF algorithm).  The main pin is a
closed form: samples 0, 1, ..., 998 plus one outlier.  Their sums are exact
integers in FP64, so the line fitted after the outlier's rejection is exactly
slope 1, the outlier and its h = 5 neighbours below it are rejected (ngood =
994), and the limits follow by hand from the median 499.5, c = 499 and the
contrast: (0, 2503.5) at contrast 0.25 and (1.5, 1000.5) at contrast 1.  This
pins the median, the (c - 1) and (npix - c) factors, the contrast, the growth of
rejections and the stopping rule.  Further pins: affine equivariance, the
degenerate sample counts, the sampling stride and the rejection of bright
outliers."""
import numpy as np
import pytest


def _ramp_with_outlier():
    img = np.full((20, 100), np.nan, np.float32)   # 2000 px: stride 2 for 1000 samples
    f = img.ravel()
    f[0:2000:2] = np.arange(1000, dtype=np.float32)
    f[1998] = 1e6
    return img


@pytest.mark.parametrize("contrast,z", [(0.25, (0.0, 2503.5)), (1.0, (1.5, 1000.5))])
def test_closed_form(orc, contrast, z):
    z1, z2, (npix, ngood) = orc.zscale(_ramp_with_outlier(), contrast=contrast)
    assert (z1, z2) == z and npix == 1000 and ngood == 994


def test_affine_equivariance(orc):
    rng = np.random.default_rng(3)
    sky = rng.normal(500.0, 20.0, (300, 400))
    sky[rng.random(sky.shape) < 0.03] = 5e4
    sky = sky.astype(np.float32)
    z1, z2, c = orc.zscale(sky)
    # a power-of-two scale and an offset that keeps every float32 sample exact
    w1, w2, cw = orc.zscale(np.float32(4.0) * sky - np.float32(1024.0))
    assert cw == c
    assert w1 == pytest.approx(4.0 * z1 - 1024.0, rel=1e-9) and w2 == pytest.approx(4.0 * z2 - 1024.0, rel=1e-9)


def test_bright_outliers_are_rejected(orc):
    rng = np.random.default_rng(5)
    sky = rng.normal(500.0, 20.0, (512, 512)).astype(np.float32)
    stars = rng.random(sky.shape) < 0.03
    sky[stars] = rng.uniform(1e4, 1e5, stars.sum()).astype(np.float32)
    z1, z2, (npix, ngood) = orc.zscale(sky)
    assert 350.0 < z1 < 500.0 < z2 < 700.0          # the sky, not the stars
    assert ngood < npix - 25                          # the ~30 star samples and their neighbours
    assert sky.max() > 1e4


def test_degenerate_counts_and_sampling(orc):
    # fewer than five samples: no fit, the sample range
    img = np.array([[3.0, np.nan, 1.0, 7.0]], np.float32)
    assert orc.zscale(img) == (1.0, 7.0, (3, 3))
    assert orc.zscale(np.array([[2.5]], np.float32)) == (2.5, 2.5, (1, 1))
    with pytest.raises(ValueError):
        orc.zscale(np.full((3, 3), np.nan, np.float32))
    # a frame smaller than n_samples is sampled whole; NaNs are dropped, not replaced
    rng = np.random.default_rng(8)
    img = rng.normal(0, 1, (20, 30)).astype(np.float32)
    img[0, :7] = np.nan
    assert orc.zscale(img)[2][0] == 600 - 7
    # stride: 10,000 px and 1000 samples take every tenth pixel
    img = np.arange(10000, dtype=np.float32).reshape(100, 100)
    z1, z2, (npix, _) = orc.zscale(img, contrast=1.0)
    assert npix == 1000
    # samples 0, 10, ..., 9990 lie on a line of slope 10 per sample: no rejection
    # (exact sums), median 4995, c = 499: z1 = 4995 - 498 * 10, z2 = min(9990, 4995 + 501 * 10)
    assert (z1, z2) == (4995.0 - 4980.0, 9990.0)

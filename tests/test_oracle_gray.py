"""Pins of the oracle's gray-scale maps (Sec. 2.2.6: value-to-gray functions
and histogram equalisation; the functions are the stated readings): closed
forms of the linear, log, power and exp scales, clipping, and the defining
property of equalisation -- the equalised values of a continuous image are
uniformly distributed -- plus monotonicity and the degenerate cases."""
import math

import numpy as np
import pytest


def test_scales_closed_forms(orc):
    x = np.array([[-5.0, 0.0, 5.0, 10.0, 15.0, np.nan]], np.float32)
    lin = orc.gray_transform(x, orc.GRAY_LINEAR, 0.0, 10.0)
    assert np.array_equal(lin[0], [0.0, 0.0, 0.5, 1.0, 1.0, 0.0])
    lg = orc.gray_transform(x, orc.GRAY_LOG, 0.0, 10.0, a=1000.0)
    assert lg[0, 2] == pytest.approx(math.log10(501.0) / math.log10(1001.0), rel=1e-14)
    assert lg[0, 1] == 0.0 and lg[0, 3] == pytest.approx(1.0, rel=1e-15)
    pw = orc.gray_transform(x, orc.GRAY_POWER, 0.0, 10.0, a=2.0)
    assert pw[0, 2] == 0.25 and pw[0, 3] == 1.0
    ex = orc.gray_transform(x, orc.GRAY_EXP, 0.0, 10.0, a=1000.0)
    assert ex[0, 2] == pytest.approx((math.sqrt(1000.0) - 1.0) / 999.0, rel=1e-14)
    assert ex[0, 1] == 0.0 and ex[0, 3] == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("law,tol", [("normal", 2e-3), ("lognormal", 1e-2)])
def test_equalised_values_are_uniform(orc, law, tol):
    """continuous images: the equalised values have the uniform distribution to
    the resolution of the fixed-width bins (the largest bin holds ~0.1% of a
    normal image's pixels with 4096 bins, ~0.5% of the skewed log-normal's)."""
    rng = np.random.default_rng(4)
    g = rng.normal(0, 1.0, (300, 400))
    img = (g if law == "normal" else np.exp(g)).astype(np.float32)
    y = orc.hist_equalize(img, nbins=4096)
    q = np.quantile(y, np.linspace(0.05, 0.95, 19))
    assert np.all(np.abs(q - np.linspace(0.05, 0.95, 19)) < tol)
    # monotone: the order of the pixels is kept
    o = np.argsort(img.ravel(), kind="stable")
    assert np.all(np.diff(y.ravel()[o]) >= -1e-15)
    assert y.min() > 0.0 and y.max() == 1.0


def test_equalising_a_ramp_is_the_identity(orc):
    """a linear ramp of distinct values fills every bin equally: the CDF is
    linear and so is the map (to half a bin)."""
    nb = 256
    img = np.linspace(0.0, 1.0, nb * 64, dtype=np.float32).reshape(64, nb)
    y = orc.hist_equalize(img, nbins=nb)
    assert np.all(np.abs(y - img) <= 1.0 / nb + 1e-6)


def test_equalise_degenerate_cases(orc):
    flat = np.full((10, 10), 3.0, np.float32)
    assert not orc.hist_equalize(flat).any()
    img = np.array([[1.0, np.inf, 2.0, np.nan]], np.float32)
    y = orc.hist_equalize(img, nbins=16)
    assert y[0, 1] == 0.0 and y[0, 3] == 0.0 and y[0, 0] == 0.5 and y[0, 2] == 1.0

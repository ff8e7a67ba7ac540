"""Pins of the oracle's detection on the smoothed frame (the 3 x 3 pyramid
detection filter of SExtractor-style pipelines; reading: weights renormalised
inside the frame, threshold unchanged): against scipy's convolution (a library
special case), a constant frame, a single bright pixel and the threshold
identity at mesh scale."""
import numpy as np
import pytest
from scipy import ndimage

K3 = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], np.float64)


def _smoothed(sub):
    """normalised convolution: the kernel over the in-frame taps only."""
    num = ndimage.convolve(sub.astype(np.float64), K3, mode="constant", cval=0.0)
    den = ndimage.convolve(np.ones_like(sub, np.float64), K3, mode="constant", cval=0.0)
    return num / den


def test_filtered_threshold_matches_normalised_convolution(orc):
    rng = np.random.default_rng(11)
    sub = rng.normal(0, 3, (37, 53)).astype(np.float32)
    sub[10:14, 20:25] += 25
    rms = np.full((3, 4), 2.0, np.float32)
    m = orc.threshold(sub, rms, 16, k=1.5, filtered=True)
    ref = _smoothed(sub) > 1.5 * 2.0
    # the oracle's rms map is the Keys interpolation of a constant grid: exactly 2
    assert np.array_equal(m.astype(bool), ref)


def test_constant_frame_and_single_pixel(orc):
    rms = np.full((2, 2), 1.0, np.float32)
    flat = np.full((20, 30), 5.0, np.float32)
    assert orc.threshold(flat, rms, 16, k=4.9, filtered=True).all()      # 5 > 4.9 everywhere, edges too
    assert not orc.threshold(flat, rms, 16, k=5.0, filtered=True).any()  # 5 > 5 nowhere
    one = np.zeros((20, 30), np.float32)
    one[10, 15] = 160.0  # smoothed: 40 at the centre, 20 at edge neighbours, 10 at corners
    m = orc.threshold(one, rms, 16, k=15.0, filtered=True)
    assert m.sum() == 5 and m[10, 15] and m[9, 15] and m[11, 15] and m[10, 14] and m[10, 16]
    m = orc.threshold(one, rms, 16, k=25.0, filtered=True)
    assert m.sum() == 1 and m[10, 15]
    # unsmoothed detection of the same frame keeps only the bright pixel
    assert orc.threshold(one, rms, 16, k=5.0).sum() == 1

"""Pins of the oracle's deblending (Sec. 2.2.5: multi-level thresholds between a
candidate's threshold and its peak, a tree of sub-components, pruning on
intensity; the stated reading for the levels, the pruning rule and the
assignment of the remaining pixels) against scenes whose answer is fixed by
construction: separated and blended stellar pairs, the contrast cut, triple
systems, a flat plateau, and the partition / numbering / translation invariants."""
import math

import numpy as np
import pytest
from scipy.special import erf


def _cdf(t):
    return 0.5 * (1.0 + erf(t / math.sqrt(2.0)))


def _stars(H, W, stars, sky_noise=0.0, seed=0):
    """pixel-integrated circular Gaussians (x, y, F, sigma)."""
    img = np.zeros((H, W))
    j, i = np.arange(W), np.arange(H)
    for x, y, F, s in stars:
        ex = _cdf((j + 0.5 - x) / s) - _cdf((j - 0.5 - x) / s)
        ey = _cdf((i + 0.5 - y) / s) - _cdf((i - 0.5 - y) / s)
        img += F * ey[:, None] * ex[None, :]
    if sky_noise:
        img += np.random.default_rng(seed).normal(0, sky_noise, img.shape)
    return img.astype(np.float32)


def _run(orc, img, cut, mincont=0.005, min_area=1):
    labels, K, _ = orc.label((img > cut).astype(np.uint8), img, min_area=min_area)
    out, K2 = orc.deblend(img, labels, K, mincont=mincont)
    return labels, K, out, K2


def _check_partition(labels, out, K2):
    # every candidate pixel gets exactly one object, nothing else does
    assert np.array_equal(out > 0, labels > 0)
    # each object lies inside one candidate
    for o in range(1, K2 + 1):
        assert len(np.unique(labels[out == o])) == 1
    # numbering: candidate by candidate, within one by raster order of first pixels
    keys = [(labels.ravel()[np.flatnonzero(out.ravel() == o)[0]], np.flatnonzero(out.ravel() == o)[0])
            for o in range(1, K2 + 1)]
    assert keys == sorted(keys)


def test_single_star_stays_whole(orc):
    img = _stars(41, 41, [(20.3, 19.6, 1e5, 1.5)])
    labels, K, out, K2 = _run(orc, img, 5.0)
    assert K == 1 and K2 == 1
    assert np.array_equal(out, labels)


def test_blended_pair_splits_and_keeps_fluxes(orc):
    """two equal stars 6 px apart (4 sigma): one candidate above 5 ADU, two
    objects, each holding its star's flux to a few per cent."""
    F = 1e5
    img = _stars(41, 51, [(21.0, 20.0, F, 1.5), (27.0, 20.5, F, 1.5)])
    labels, K, out, K2 = _run(orc, img, 5.0)
    assert K == 1 and K2 == 2
    _check_partition(labels, out, K2)
    f = [img[out == o].sum() for o in (1, 2)]
    assert f[0] == pytest.approx(F, rel=0.03) and f[1] == pytest.approx(F, rel=0.03)
    # each object holds its own peak
    assert out[20, 21] != out[20, 27]


def test_contrast_cut(orc):
    """a companion with 10% of the main star's flux, 10 px away: the two separate
    at the lowest levels, where the companion's branch holds nearly all of its
    flux (~9% of the candidate's), so it splits at mincont = 0.05 and stays
    merged at mincont = 0.2."""
    img = _stars(41, 61, [(20.0, 20.0, 1e5, 1.5), (30.0, 20.0, 1e4, 1.5)])
    labels, K, _, _ = _run(orc, img, 0.5)
    assert K == 1
    _, K_low = orc.deblend(img, labels, K, mincont=0.05)
    _, K_high = orc.deblend(img, labels, K, mincont=0.2)
    assert K_low == 2 and K_high == 1


def test_triple_and_separate_candidates(orc):
    img = _stars(60, 80, [(20.0, 20.0, 1e5, 1.4), (26.0, 21.0, 8e4, 1.4), (23.0, 26.0, 6e4, 1.4),
                          (60.0, 40.0, 5e4, 1.4)])
    labels, K, out, K2 = _run(orc, img, 5.0)
    assert K == 2 and K2 == 4
    _check_partition(labels, out, K2)
    # the isolated star is untouched (its candidate keeps one object)
    iso = labels[40, 60]
    assert len(np.unique(out[labels == iso])) == 1


def test_flat_plateau_is_not_split(orc):
    """P = T: no levels, the candidate stays whole."""
    img = np.zeros((20, 20), np.float32)
    img[5:12, 4:15] = 10.0
    labels, K, out, K2 = _run(orc, img, 1.0)
    assert K == 1 and K2 == 1 and np.array_equal(out, labels)


def test_saddle_between_two_peaks(orc):
    """two 1-D ridges of height 100 joined by a saddle at 20 on a plateau of 10:
    every level between 20 and 100 holds two nodes, so the pair splits and the
    saddle pixels go to the nearer, equal-looking peak by likelihood."""
    img = np.full((5, 21), 10.0, np.float32)
    prof = np.array([10, 30, 60, 100, 60, 30, 20, 30, 60, 100, 60, 30, 10, 10, 10, 10, 10, 10, 10, 10, 10],
                    np.float32)
    img[2, :] = prof
    labels, K, out, K2 = _run(orc, img, 5.0)
    assert K == 1 and K2 == 2
    _check_partition(labels, out, K2)
    assert out[2, 3] != out[2, 9]


def test_translation_invariance_and_noise(orc):
    img = _stars(64, 64, [(25.0, 30.0, 5e4, 1.6), (31.0, 31.0, 3e4, 1.6), (45.0, 12.0, 2e4, 1.6)],
                 sky_noise=3.0, seed=4)
    labels, K, out, K2 = _run(orc, img, 10.0, min_area=5)
    big = np.zeros((80, 90), np.float32)
    big[9:73, 17:81] = img
    lab2 = np.zeros((80, 90), np.int32)
    lab2[9:73, 17:81] = labels
    out2, K3 = orc.deblend(big, lab2, K)
    assert K3 == K2
    assert np.array_equal(out2[9:73, 17:81], out)
    _check_partition(labels, out, K2)

"""Pins of the oracle's detection steps (Sec. 2.2.5: pixel detection above a
threshold, connection into candidates, per-candidate peak / total flux) against
scipy.ndimage and exhaustive small cases."""
import numpy as np
import pytest
from scipy import ndimage


def _scipy_label(mask, min_area):
    """Library reference: 8-connected labels (scipy numbers components in raster
    order of their first pixel), small ones dropped, survivors renumbered."""
    lab, n = ndimage.label(mask, structure=np.ones((3, 3), int))
    if n == 0:
        return lab, 0
    area = np.bincount(lab.ravel(), minlength=n + 1)
    keep = np.zeros(n + 1, np.int64)
    kk = 0
    for c in range(1, n + 1):
        if area[c] >= min_area:
            kk += 1
            keep[c] = kk
    return keep[lab].astype(np.int32), kk


def test_threshold_strict(orc):
    """detected iff sub > k * rms (strict), rms interpolated (here constant)."""
    rms = np.full((2, 2), 2.0, np.float32)
    sub = np.array([[3.0, 2.999999, 3.000001, -5.0]] * 4, np.float32)
    m = orc.threshold(sub, rms, 2, k=1.5)
    assert m[:, 0].sum() == 0 and m[:, 1].sum() == 0 and m[:, 2].all() and not m[:, 3].any()
    m = orc.threshold(sub, rms, 2, k=1.5, thresh_abs=4.0)
    assert m.sum() == 0


def test_label_vs_scipy_random(orc):
    rng = np.random.default_rng(0)
    for trial in range(30):
        H, W = rng.integers(1, 40, 2)
        p = rng.uniform(0.05, 0.7)
        mask = (rng.uniform(size=(H, W)) < p).astype(np.uint8)
        sub = rng.uniform(0.1, 5.0, (H, W)).astype(np.float32)
        for min_area in (1, 3, 5):
            lab, K, _ = orc.label(mask, sub, min_area)
            ref, Kr = _scipy_label(mask, min_area)
            assert K == Kr
            assert np.array_equal(lab, ref)


def test_label_exhaustive_4x4(orc):
    """All 65,536 binary 4x4 masks, min_area 1 and 3."""
    bits = (np.arange(1 << 16)[:, None] >> np.arange(16)[None, :]) & 1
    sub = np.ones((4, 4), np.float32)
    for min_area in (1, 3):
        for code in range(1 << 16):
            mask = bits[code].reshape(4, 4).astype(np.uint8)
            lab, K, _ = orc.label(mask, sub, min_area)
            ref, Kr = _scipy_label(mask, min_area)
            if K != Kr or not np.array_equal(lab, ref):
                pytest.fail(f"mismatch for mask code {code} min_area {min_area}")


def test_label_stats_vs_scipy(orc):
    rng = np.random.default_rng(1)
    H, W = 60, 75
    mask = (rng.uniform(size=(H, W)) < 0.3).astype(np.uint8)
    sub = rng.uniform(0.5, 10.0, (H, W)).astype(np.float32)
    lab, K, st = orc.label(mask, sub, 4)
    idx = np.arange(1, K + 1)
    s64 = sub.astype(np.float64)
    assert np.array_equal(st["area"], ndimage.sum_labels(np.ones_like(s64), lab, idx).astype(int))
    assert np.allclose(st["sum"], ndimage.sum_labels(s64, lab, idx), rtol=1e-13)
    assert np.array_equal(st["peak"], ndimage.maximum(s64, lab, idx))
    com = np.array(ndimage.center_of_mass(s64, lab, idx))
    assert np.allclose(st["ybar"], com[:, 0], rtol=1e-12)
    assert np.allclose(st["xbar"], com[:, 1], rtol=1e-12)
    for k, sl in enumerate(ndimage.find_objects(lab)):
        assert (st["ymin"][k], st["ymax"][k] + 1) == (sl[0].start, sl[0].stop)
        assert (st["xmin"][k], st["xmax"][k] + 1) == (sl[1].start, sl[1].stop)
        first = np.flatnonzero(lab.ravel() == k + 1)[0]
        assert st["first"][k] == first
    # numbering is monotone in the first-pixel raster index
    assert np.all(np.diff(st["first"]) > 0)


def test_label_capacity(orc):
    """K counts every survivor; stats are kept for the first max_src only."""
    mask = np.zeros((5, 20), np.uint8)
    mask[:, ::2] = 1          # 10 vertical bars of area 5
    sub = np.ones(mask.shape, np.float32)
    lab, K, st = orc.label(mask, sub, 5, max_src=4)
    assert K == 10 and len(st["area"]) == 4 and lab.max() == 10
    assert list(st["first"]) == [0, 2, 4, 6]


def test_label_empty_and_full(orc):
    sub = np.ones((7, 9), np.float32)
    lab, K, _ = orc.label(np.zeros((7, 9), np.uint8), sub, 1)
    assert K == 0 and lab.max() == 0
    lab, K, st = orc.label(np.ones((7, 9), np.uint8), sub, 5)
    assert K == 1 and np.all(lab == 1) and st["area"][0] == 63

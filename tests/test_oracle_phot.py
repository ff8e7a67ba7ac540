"""Pins of the oracle's per-source steps: windowed centroid, exact pixel/circle
overlap, sky annulus and aperture flux (Sec. 2.2.5 photometry and positions,
with the stated readings), against geometry, closed forms and brute force."""
import math

import numpy as np
import pytest
from scipy.special import erf


def _gauss_frame(H, W, x, y, F, fwhm):
    """noise-free pixel-integrated circular Gaussian (normal-CDF differences)."""
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    j = np.arange(W)
    i = np.arange(H)
    cdf = lambda t: 0.5 * (1.0 + erf(t / math.sqrt(2.0)))
    ex = cdf((j + 0.5 - x) / s) - cdf((j - 0.5 - x) / s)
    ey = cdf((i + 0.5 - y) / s) - cdf((i - 0.5 - y) / s)
    return (F * ey[:, None] * ex[None, :]).astype(np.float32)


# ----------------------------------------------------------------- overlap
def test_overlap_sum_is_disk_area(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        cx, cy = rng.uniform(20, 21, 2)
        r = rng.uniform(0.3, 7.0)
        tot = 0.0
        for i in range(int(cy - r) - 2, int(cy + r) + 3):
            for j in range(int(cx - r) - 2, int(cx + r) + 3):
                tot += orc.overlap(cx, cy, r, j - 0.5, j + 0.5, i - 0.5, i + 0.5)
        assert tot == pytest.approx(math.pi * r * r, rel=1e-12)


def test_overlap_special_cases(orc):
    r = 3.0
    assert orc.overlap(0, 0, r, -1, 1, -1, 1) == pytest.approx(4.0, abs=1e-14)      # box inside disk
    assert orc.overlap(0, 0, 0.4, -0.5, 0.5, -0.5, 0.5) == pytest.approx(math.pi * 0.16, rel=1e-14)
    assert orc.overlap(0, 0, r, 0, 10, -10, 10) == pytest.approx(math.pi * 9 / 2, rel=1e-14)
    assert orc.overlap(0, 0, r, 0, 10, 0, 10) == pytest.approx(math.pi * 9 / 4, rel=1e-14)
    assert orc.overlap(0, 0, r, 3.0, 4.0, -1, 1) == 0.0
    assert orc.overlap(0, 0, r, 5, 6, 5, 6) == 0.0
    # circular segment cut by the line x = a: r^2 acos(a/r) - a sqrt(r^2 - a^2)
    a = 1.7
    seg = r * r * math.acos(a / r) - a * math.sqrt(r * r - a * a)
    assert orc.overlap(0, 0, r, a, 10, -10, 10) == pytest.approx(seg, rel=1e-13)


def test_overlap_symmetry(orc):
    rng = np.random.default_rng(4)
    for _ in range(50):
        cx, cy, r = rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.2, 3)
        x0, y0 = rng.uniform(-3, 2, 2)
        x1, y1 = x0 + 1, y0 + 1
        a = orc.overlap(cx, cy, r, x0, x1, y0, y1)
        assert orc.overlap(-cx, cy, r, -x1, -x0, y0, y1) == pytest.approx(a, abs=1e-13)
        assert orc.overlap(cy, cx, r, y0, y1, x0, x1) == pytest.approx(a, abs=1e-13)
        assert orc.overlap(cx, -cy, r, x0, x1, -y1, -y0) == pytest.approx(a, abs=1e-13)


def test_overlap_vs_supersampling(orc):
    """Brute force: fraction of an n x n grid of sub-pixel centres inside the
    circle; its error is below ~ (chord length) / n."""
    rng = np.random.default_rng(5)
    n = 1500
    t = (np.arange(n) + 0.5) / n - 0.5
    for _ in range(12):
        cx, cy = rng.uniform(-0.5, 0.5, 2)
        r = rng.uniform(0.3, 3.0)
        i, j = rng.integers(-3, 4, 2)
        inside = ((j + t[None, :] - cx) ** 2 + (i + t[:, None] - cy) ** 2) < r * r
        bf = inside.mean()
        ex = orc.overlap(cx, cy, r, j - 0.5, j + 0.5, i - 0.5, i + 0.5)
        assert abs(bf - ex) < 3.0 / n


# ---------------------------------------------------------------- centroid
def test_centroid_exact_on_symmetric_star(orc):
    H = W = 41
    for (x, y) in [(20.0, 20.0), (20.5, 19.5), (17.0, 23.5)]:
        img = _gauss_frame(H, W, x, y, 1e4, 3.0)
        cx, cy, it, fl = orc.centroid(img, [x + 0.3], [y - 0.2])
        assert fl[0] == 0
        assert cx[0] == pytest.approx(x, abs=1e-5) and cy[0] == pytest.approx(y, abs=1e-5)


def test_centroid_subpixel_truth(orc):
    rng = np.random.default_rng(6)
    H = W = 41
    for _ in range(10):
        x, y = rng.uniform(18, 22, 2)
        img = _gauss_frame(H, W, x, y, 1e4, rng.uniform(2.5, 4.0))
        cx, cy, it, fl = orc.centroid(img, [round(x)], [round(y)])
        assert fl[0] == 0
        assert abs(cx[0] - x) < 1e-2 and abs(cy[0] - y) < 1e-2


def test_centroid_integer_translation(orc):
    rng = np.random.default_rng(8)
    img = rng.normal(0, 1, (50, 60)).astype(np.float32)
    img += _gauss_frame(50, 60, 20.3, 21.7, 3e3, 3.0)
    a = orc.centroid(img, [20.0], [22.0])
    img2 = np.zeros((50, 60), np.float32)
    img2[3:, 5:] = img[:-3, :-5]
    b = orc.centroid(img2, [25.0], [25.0])
    assert b[0][0] - 5 == pytest.approx(a[0][0], abs=1e-9)
    assert b[1][0] - 3 == pytest.approx(a[1][0], abs=1e-9)


def test_centroid_nonpositive_window_keeps_seed(orc):
    img = -np.ones((30, 30), np.float32)
    x, y, it, fl = orc.centroid(img, [14.25], [15.5])
    assert (x[0], y[0]) == (14.25, 15.5) and fl[0] & 2


def test_centroid_edge_flag(orc):
    img = _gauss_frame(30, 30, 1.0, 15.0, 1e4, 3.0)
    x, y, it, fl = orc.centroid(img, [1.0], [15.0])
    assert fl[0] & 1


# --------------------------------------------------------------- aperture
def test_aperture_flat_sky(orc):
    img = np.full((60, 60), 42.5, np.float32)
    ph = orc.aperture(img, [30.3], [29.8])
    assert ph["sky"][0] == 42.5
    assert ph["flux"][0] == pytest.approx(0.0, abs=1e-10)
    assert ph["area"][0] == pytest.approx(math.pi * 25, rel=1e-12)
    assert ph["flags"][0] == 0


def test_aperture_annulus_count_brute(orc):
    """number of pixel centres with 8 <= d < 12, counted directly on a lattice."""
    rng = np.random.default_rng(9)
    img = np.zeros((80, 80), np.float32)
    for _ in range(10):
        x, y = rng.uniform(30, 50, 2).astype(np.float32)
        ph = orc.aperture(img, [x], [y])
        jj, ii = np.meshgrid(np.arange(80), np.arange(80))
        d2 = (jj - np.float64(x)) ** 2 + (ii - np.float64(y)) ** 2
        assert ph["n_ann"][0] == int(((d2 >= 64) & (d2 < 144)).sum())


def test_aperture_gaussian_closed_form(orc):
    """Noise-free pixel-integrated Gaussian, FWHM 3, r = 5: the disk holds
    F (1 - exp(-r^2 / 2 sigma^2)) = 0.999548 F.  Weighting pixel-integrated values
    by their overlap area under-counts the inner (brighter) part of the edge
    pixels; for this profile that first-order pixelisation term is -4.5e-4 F, so
    the pin allows 6e-4 (an aperture of r = 4.8 would already miss it)."""
    rng = np.random.default_rng(10)
    s = 3.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    frac = 1 - math.exp(-25 / (2 * s * s))
    assert frac == pytest.approx(0.999548, abs=1e-6)
    for _ in range(5):
        x, y = rng.uniform(40, 41, 2)
        img = _gauss_frame(81, 81, x, y, 1e5, 3.0)
        ph = orc.aperture(img, [x], [y])
        assert abs(ph["flux"][0] / 1e5 - frac) < 6e-4
        assert ph["sky"][0] == pytest.approx(0.0, abs=1e-6)


def test_aperture_piecewise_constant_exact(orc):
    """On a flat sky c plus one raised pixel, flux = (raised value) x (its
    overlap with the disk), whatever the pixel: inner pixels count fully, outer
    ones not at all, edge pixels by their exact area."""
    c = 10.0
    for (i, j, w_expect) in [(30, 30, 1.0), (30, 34, 1.0), (30, 37, 0.0), (25, 25, 0.0)]:
        img = np.full((61, 61), c, np.float32)
        img[i, j] += 1000.0
        ph = orc.aperture(img, [30.0], [30.0])
        assert ph["sky"][0] == c
        assert ph["flux"][0] == pytest.approx(1000.0 * w_expect, abs=1e-9)
    img = np.full((61, 61), c, np.float32)
    img[30, 35] += 1000.0     # centre at distance 5: straddles the edge
    ph = orc.aperture(img, [30.0], [30.0])
    w = orc.overlap(30, 30, 5, 34.5, 35.5, 29.5, 30.5)
    assert 0.3 < w < 0.7 and ph["flux"][0] == pytest.approx(1000.0 * w, rel=1e-12)


def test_aperture_edge_and_few(orc):
    img = np.ones((20, 20), np.float32)
    ph = orc.aperture(img, [1.0], [1.0])
    assert ph["flags"][0] & 1
    ph = orc.aperture(img, [10.0], [10.0], r_in=8, r_out=8.5, min_ann=200)
    assert ph["flags"][0] & 4 and ph["sky"][0] == 0.0


def test_overlap_sum_is_disk_area_on_edge_lines(orc):
    """centres on pixel edge lines and centres, where an integer radius makes
    the circle touch a pixel edge line at a single point: the weights still add
    up to pi r^2 (the tangent point splits the chord integral)."""
    for r in (3.0, 5.0, 4.5):
        for cx, cy in [(0.0, 0.5), (0.5, 0.0), (0.0, 0.0), (0.5, 0.5), (0.25, 0.5), (0.5, 0.75)]:
            tot = sum(orc.overlap(cx, cy, r, j - 0.5, j + 0.5, i - 0.5, i + 0.5)
                      for i in range(-8, 9) for j in range(-8, 9))
            assert tot == pytest.approx(math.pi * r * r, rel=1e-12), (r, cx, cy)

"""Pins of the oracle's auto (Kron) photometry (Sec. 2.2.5 lists auto photometry;
the method is the stated reading: footprint moments, Kron first-moment radius,
elliptical aperture max(2.5 r1, 3.5)) against closed forms of a pixel-integrated
Gaussian, a single-pixel source and invariants under translation, transposition
and scaling."""
import math

import numpy as np
import pytest
from scipy.special import erf

# E[r] of a 2-D normal in units of its sigma: sqrt(pi/2)
KRON_GAUSS = math.sqrt(math.pi / 2.0)
# fraction of a 2-D normal inside Mahalanobis radius 3.5
FRAC_35 = 1.0 - math.exp(-3.5 ** 2 / 2.0)


def _cdf(t):
    return 0.5 * (1.0 + erf(t / math.sqrt(2.0)))


def _elliptical_gauss(H, W, x, y, F, sx, sy, th, sub=8):
    """noise-free elliptical Gaussian integrated over each pixel by sub x sub
    point samples of the exact profile (circular case: erf products)."""
    if sx == sy:
        j, i = np.arange(W), np.arange(H)
        ex = _cdf((j + 0.5 - x) / sx) - _cdf((j - 0.5 - x) / sx)
        ey = _cdf((i + 0.5 - y) / sy) - _cdf((i - 0.5 - y) / sy)
        return F * ey[:, None] * ex[None, :]
    off = (np.arange(sub) + 0.5) / sub - 0.5
    xs = (np.arange(W)[:, None] + off[None, :]).ravel()
    ys = (np.arange(H)[:, None] + off[None, :]).ravel()
    dx, dy = xs[None, :] - x, ys[:, None] - y
    c, s = math.cos(th), math.sin(th)
    u, v = c * dx + s * dy, -s * dx + c * dy
    p = F / (2 * math.pi * sx * sy) * np.exp(-0.5 * (u * u / sx ** 2 + v * v / sy ** 2))
    return p.reshape(H, sub, W, sub).mean(axis=(1, 3))


def _source(orc, f, cut):
    """label the single footprint f > cut with the oracle's own labeling."""
    f = f.astype(np.float32)
    labels, K, st = orc.label((f > cut).astype(np.uint8), f, min_area=1)
    assert K == 1
    return f, labels, st


def test_circular_gaussian_closed_forms(orc):
    s, F = 5.0, 1e6
    f = _elliptical_gauss(101, 101, 50.3, 49.7, F, s, s, 0.0)
    sub, labels, st = _source(orc, f, 1e-7 * f.max())
    a = orc.auto_phot(sub, labels, st)
    # binning a normal adds 1/12 to its variance (Sheppard)
    assert a["x2"][0] == pytest.approx(s * s + 1 / 12, rel=2e-3)
    assert a["y2"][0] == pytest.approx(s * s + 1 / 12, rel=2e-3)
    assert abs(a["xy"][0]) < 1e-3
    assert a["kron"][0] == pytest.approx(KRON_GAUSS, rel=5e-3)
    # 2.5 r1 = 3.13 < 3.5: the aperture is the minimum one
    assert a["flux"][0] == pytest.approx(FRAC_35 * F, rel=1.5e-3)
    assert a["area"][0] == pytest.approx(math.pi * 3.5 ** 2 * (s * s + 1 / 12), rel=0.03)
    assert a["flags"][0] == 0


@pytest.mark.parametrize("th", [0.5, -1.1])
def test_elliptical_gaussian_moments(orc, th):
    sx, sy, F = 6.0, 3.0, 1e6
    f = _elliptical_gauss(121, 121, 60.2, 59.6, F, sx, sy, th)
    sub, labels, st = _source(orc, f, 1e-7 * f.max())
    a = orc.auto_phot(sub, labels, st)
    c, s = math.cos(th), math.sin(th)
    x2 = sx * sx * c * c + sy * sy * s * s + 1 / 12
    y2 = sx * sx * s * s + sy * sy * c * c + 1 / 12
    xy = (sx * sx - sy * sy) * s * c
    assert a["x2"][0] == pytest.approx(x2, rel=3e-3)
    assert a["y2"][0] == pytest.approx(y2, rel=3e-3)
    assert a["xy"][0] == pytest.approx(xy, rel=3e-3)
    assert a["kron"][0] == pytest.approx(KRON_GAUSS, rel=5e-3)
    assert a["flux"][0] == pytest.approx(FRAC_35 * F, rel=1.5e-3)


def test_wide_aperture_when_kron_radius_is_large(orc):
    """a flat-topped source (uniform disk of radius 6 px on zero sky): the
    moments give x2 = y2 = rho^2 / 4 and the Kron radius of a uniform disk is
    (2/3) rho / sqrt(x2) = 4/3 in moment units, so R = max(2.5 x 4/3, 3.5) = 3.5;
    a disk plus a faint wide halo pushes r1 up and the aperture to 2.5 r1."""
    H = W = 81
    yy, xx = np.mgrid[0:H, 0:W]
    d = np.hypot(xx - 40.0, yy - 40.0)
    disk = (d <= 6.0).astype(np.float64) * 100.0
    sub, labels, st = _source(orc, disk, 50.0)
    a = orc.auto_phot(sub, labels, st)
    assert a["kron"][0] == pytest.approx(4.0 / 3.0, rel=0.03)
    assert a["flux"][0] == pytest.approx(disk.sum(), rel=1e-12)
    halo = disk + 5.0 * (d < 30.0)
    sub, labels, st = _source(orc, halo, 50.0)
    b = orc.auto_phot(sub, labels, st)
    assert b["kron"][0] > 1.4
    # aperture 2.5 r1 in moment units; the flux holds every pixel inside it
    R = 2.5 * b["kron"][0]
    r2 = ((b["y2"][0] * (xx - st["xbar"][0]) ** 2 + b["x2"][0] * (yy - st["ybar"][0]) ** 2 -
           2 * b["xy"][0] * (xx - st["xbar"][0]) * (yy - st["ybar"][0])) /
          (b["x2"][0] * b["y2"][0] - b["xy"][0] ** 2))
    inside = r2 <= R * R
    assert b["area"][0] == inside.sum()
    assert b["flux"][0] == pytest.approx(halo[inside].sum(), rel=1e-12)


def test_single_pixel_source(orc):
    """a one-pixel footprint: moments 0, so x2 = y2 = 1/12 and the elliptical
    radius is d sqrt(12).  Alone, all the flux sits at r = 0: the Kron sum is 0
    (KRON_BAD) and R = 3.5, i.e. 3.5 / sqrt(12) = 1.01 px -- the pixel and its
    four edge neighbours.  A pixel 2 px away (r = 6.9) is outside both the Kron
    region (r <= 6) and the aperture; an edge neighbour (r = 3.46) is inside
    both and gives r1 = 3.46 x 7 / 107."""
    sub = np.zeros((41, 41), np.float32)
    sub[20, 20] = 100.0
    sub[20, 22] = 1000.0
    labels = np.zeros((41, 41), np.int32)
    labels[20, 20] = 1
    st = dict(xmin=[20], xmax=[20], ymin=[20], ymax=[20], xbar=[20.0], ybar=[20.0])
    a = orc.auto_phot(sub, labels, st)
    assert a["x2"][0] == 1 / 12 and a["y2"][0] == 1 / 12 and a["xy"][0] == 0
    assert a["kron"][0] == 0 and a["flags"][0] == orc.FLAG_KRON_BAD
    assert a["area"][0] == 5 and a["flux"][0] == 100.0
    sub[21, 20] = 7.0
    b = orc.auto_phot(sub, labels, st)
    assert b["kron"][0] == pytest.approx(math.sqrt(12.0) * 7.0 / 107.0, rel=1e-14)
    assert b["flags"][0] == 0 and b["area"][0] == 5 and b["flux"][0] == 107.0


def test_invariants_translation_transpose_scale(orc):
    rng = np.random.default_rng(5)
    f = _elliptical_gauss(64, 64, 30.4, 31.7, 2e4, 2.2, 1.4, 0.7) + rng.normal(0, 3, (64, 64))
    sub, labels, st = _source(orc, f, 40.0)
    a = orc.auto_phot(sub, labels, st)
    assert a["flags"][0] == 0 and a["kron"][0] > 0
    # whole-pixel translation: identical numbers
    sh = np.zeros((80, 80), np.float32)
    sh[7:71, 11:75] = sub
    lab = np.zeros((80, 80), np.int32)
    lab[7:71, 11:75] = labels
    st2 = dict(st, xmin=st["xmin"] + 11, xmax=st["xmax"] + 11, ymin=st["ymin"] + 7,
               ymax=st["ymax"] + 7, xbar=st["xbar"].astype(np.float32) + 11,
               ybar=st["ybar"].astype(np.float32) + 7)
    b = orc.auto_phot(sh, lab, st2)
    for k in ("flux", "area", "kron", "x2", "y2", "xy"):
        assert b[k][0] == pytest.approx(a[k][0], rel=1e-12, abs=1e-12), k
    # transpose: x and y swap roles
    st3 = dict(xmin=st["ymin"], xmax=st["ymax"], ymin=st["xmin"], ymax=st["xmax"],
               xbar=st["ybar"], ybar=st["xbar"])
    c = orc.auto_phot(np.ascontiguousarray(sub.T), np.ascontiguousarray(labels.T), st3)
    assert c["x2"][0] == pytest.approx(a["y2"][0], rel=1e-12)
    assert c["y2"][0] == pytest.approx(a["x2"][0], rel=1e-12)
    for k in ("flux", "area", "kron", "xy"):
        assert c[k][0] == pytest.approx(a[k][0], rel=1e-12), k
    # scaling by 2: flux doubles, shape and radius unchanged (powers of two are exact)
    d = orc.auto_phot(2 * sub, labels, st)
    assert d["flux"][0] == 2 * a["flux"][0]
    for k in ("kron", "x2", "y2", "xy", "area"):
        assert d[k][0] == a[k][0], k


def test_edge_flag_and_in_frame_sum(orc):
    f = _elliptical_gauss(40, 40, 2.2, 20.0, 1e4, 1.5, 1.5, 0.0)
    sub, labels, st = _source(orc, f, 1.0)
    a = orc.auto_phot(sub, labels, st)
    assert a["flags"][0] & orc.FLAG_EDGE
    # the in-frame part of the aperture: recount directly
    yy, xx = np.mgrid[0:40, 0:40]
    dx, dy = xx - np.float32(st["xbar"][0]), yy - np.float32(st["ybar"][0])
    det = a["x2"][0] * a["y2"][0] - a["xy"][0] ** 2
    r2 = (a["y2"][0] * dx * dx - 2 * a["xy"][0] * dx * dy + a["x2"][0] * dy * dy) / det
    R = max(2.5 * a["kron"][0], 3.5)
    assert a["area"][0] == (r2 <= R * R).sum()

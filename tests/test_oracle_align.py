"""Pins of the oracle's image alignment (Sec. 2.2.3: Eqs. 5-7, their inverse
chain, the partial affine estimate and bilinear reprojection).  Each pin rests on
something other than the oracle's own formulas: the tangent point maps to CRVAL;
the gnomonic projection's closed forms (the angular distance from the tangent
point is atan of the radial standard coordinate, and lines through the reference
pixel map to great circles), checked with spherical trigonometry written here;
a SIP term equals a shift of the input pixel; the inverse chain undoes the
forward one; the similarity fit recovers a known transform and agrees with
numpy's least squares; bilinear reprojection is exact for translations and for
linear ramps."""
import math

import numpy as np
import pytest

D2R = math.pi / 180.0


def _wcs(crpix=(1024.5, 1024.5), crval=(150.0, 30.0), scale=1.0 / 3600, rot=0.0, a=None, b=None, order=0):
    c, s = math.cos(rot), math.sin(rot)
    cd = [[-scale * c, scale * s], [scale * s, scale * c]]
    w = dict(crpix=crpix, crval=crval, cd=cd, a_order=order, b_order=order)
    if a is not None:
        w["a"] = a
    if b is not None:
        w["b"] = b
    return w


def _unit(ra, dec):
    ra, dec = np.asarray(ra) * D2R, np.asarray(dec) * D2R
    return np.stack([np.cos(dec) * np.cos(ra), np.cos(dec) * np.sin(ra), np.sin(dec)], -1)


def _sep(ra1, de1, ra2, de2):
    """angular separation (radians) from unit vectors: atan2(|u x v|, u . v)"""
    u, v = _unit(ra1, de1), _unit(ra2, de2)
    return np.arctan2(np.linalg.norm(np.cross(u, v), axis=-1), np.sum(u * v, -1))


def test_reference_pixel_maps_to_crval(orc):
    a = np.zeros((6, 6)); a[2, 0] = 3e-6; a[0, 3] = 1e-9
    w = _wcs(crpix=(500.25, 300.75), crval=(210.5, -45.25), a=a, b=a.T.copy(), order=3)
    ra, de = orc.wcs_pix2world(w, [499.25], [299.75])
    assert ra[0] == pytest.approx(210.5, abs=1e-12) and de[0] == pytest.approx(-45.25, abs=1e-12)


@pytest.mark.parametrize("crval", [(0.0, 0.0), (150.0, 30.0), (300.0, -72.5), (45.0, 89.9)])
def test_gnomonic_distance_is_atan_of_radius(orc, crval):
    """TAN projection: a point at standard-coordinate radius r (radians) lies at
    angular distance atan(r) from the tangent point, in the direction atan2(p, q)
    east of north (checked with the position angle from spherical trigonometry)."""
    scale = 20.0 / 3600  # 20 arcsec/px: a field a few degrees wide
    w = _wcs(crval=crval, scale=scale, crpix=(1.0, 1.0))
    rng = np.random.default_rng(3)
    dx, dy = rng.uniform(-2000, 2000, 50), rng.uniform(-2000, 2000, 50)
    ra, de = orc.wcs_pix2world(w, dx, dy)
    p, q = -scale * dx * D2R, scale * dy * D2R   # CD = diag(-s, s)
    r = np.hypot(p, q)
    sep = _sep(ra, de, crval[0], crval[1])
    assert np.max(np.abs(sep - np.arctan(r))) < 1e-13
    # position angle of each point seen from the tangent point, east of north
    a0, d0 = crval[0] * D2R, crval[1] * D2R
    al, dl = ra * D2R, de * D2R
    pa = np.arctan2(np.sin(al - a0) * np.cos(dl), np.cos(d0) * np.sin(dl) - np.sin(d0) * np.cos(dl) * np.cos(al - a0))
    dpa = np.angle(np.exp(1j * (pa - np.arctan2(p, q))))
    assert np.max(np.abs(dpa)) < 1e-10


def test_lines_through_reference_pixel_are_great_circles(orc):
    w = _wcs(crval=(80.0, 20.0), scale=10.0 / 3600, rot=0.3, crpix=(0.0, 0.0))
    t = np.linspace(-3000, 3000, 41)
    ra, de = orc.wcs_pix2world(w, 0.7 * t - 1.0, -0.4 * t - 1.0)
    u = _unit(ra, de)
    n = np.cross(u[0], u[-1])
    n /= np.linalg.norm(n)
    assert np.max(np.abs(u @ n)) < 1e-13


def test_sip_term_is_a_shift_of_the_input_pixel(orc):
    """xi = u + A_20 u^2 and eta = v + B_11 u v: the distorted WCS at (x, y) equals
    the undistorted one at the shifted pixel (pins the term indexing and sign)."""
    a = np.zeros((6, 6)); a[2, 0] = 2e-6
    b = np.zeros((6, 6)); b[1, 1] = -3e-6
    wd = _wcs(crpix=(1000.0, 800.0), a=a, b=b, order=2)
    w0 = _wcs(crpix=(1000.0, 800.0))
    rng = np.random.default_rng(5)
    x, y = rng.uniform(0, 2000, 30), rng.uniform(0, 1600, 30)
    u, v = x + 1 - 1000.0, y + 1 - 800.0
    r1, d1 = orc.wcs_pix2world(wd, x, y)
    r0, d0 = orc.wcs_pix2world(w0, x + 2e-6 * u * u, y - 3e-6 * u * v)
    assert np.max(_sep(r1, d1, r0, d0)) < 1e-14


@pytest.mark.parametrize("order", [0, 3, 5])
def test_inverse_chain_undoes_the_forward_chain(orc, order):
    rng = np.random.default_rng(order)
    a, b = np.zeros((6, 6)), np.zeros((6, 6))
    for p in range(6):
        for q in range(6 - p):
            if 2 <= p + q <= order:
                # a few px of distortion at the field's corners, as in survey cameras
                a[p, q] = rng.normal(0, 1.0) * 3.0 * 2048.0 ** (-p - q)
                b[p, q] = rng.normal(0, 1.0) * 3.0 * 2048.0 ** (-p - q)
    w = _wcs(crpix=(2048.5, 2048.5), crval=(12.0, -33.0), scale=1.5 / 3600, rot=0.7, a=a, b=b, order=order)
    x, y = rng.uniform(0, 4096, 200), rng.uniform(0, 4096, 200)
    ra, de = orc.wcs_pix2world(w, x, y)
    x2, y2 = orc.wcs_world2pix(w, ra, de)
    assert np.max(np.abs(x2 - x)) < 1e-8 and np.max(np.abs(y2 - y)) < 1e-8


def test_points_beyond_the_horizon_have_no_image(orc):
    w = _wcs(crval=(0.0, 0.0))
    x, y = orc.wcs_world2pix(w, [180.0, 100.0, 10.0], [0.0, 0.0, 0.0])
    assert np.isnan(x[0]) and np.isnan(x[1]) and np.isfinite(x[2])


def test_map_identity_and_translation(orc):
    a = np.zeros((6, 6)); a[3, 0] = 1e-10; a[1, 1] = 5e-6
    w = _wcs(crpix=(300.5, 200.5), crval=(33.0, 44.0), a=a, b=a.copy(), order=3)
    xo, yo = orc.wcs_map(w, w, 601, 401, step=25)
    gx, gy = np.meshgrid(np.arange(0, 601, 25.0), np.arange(0, 401, 25.0))
    assert xo.shape == (17, 25) and np.max(np.abs(xo - gx)) < 1e-8 and np.max(np.abs(yo - gy)) < 1e-8
    w0, w1 = _wcs(crpix=(300.5, 200.5)), _wcs(crpix=(310.5, 190.5))
    xo, yo = orc.wcs_map(w0, w1, 601, 401, step=50)
    gx, gy = np.meshgrid(np.arange(0, 601, 50.0), np.arange(0, 401, 50.0))
    assert np.max(np.abs(xo - gx - 10.0)) < 1e-9 and np.max(np.abs(yo - gy + 10.0)) < 1e-9


def test_affine_fit_recovers_a_similarity_and_matches_lstsq(orc):
    rng = np.random.default_rng(9)
    x, y = rng.uniform(0, 4000, 500), rng.uniform(0, 4000, 500)
    s, th, tx, ty = 0.98, 0.013, 12.5, -7.25
    xt = s * (math.cos(th) * x - math.sin(th) * y) + tx
    yt = s * (math.sin(th) * x + math.cos(th) * y) + ty
    M, Mi = orc.affine_fit(x, y, xt, yt)
    ref = np.array([[s * math.cos(th), -s * math.sin(th), tx], [s * math.sin(th), s * math.cos(th), ty]])
    assert np.max(np.abs(M - ref)) < 1e-10
    comp = np.vstack([Mi, [0, 0, 1]]) @ np.vstack([M, [0, 0, 1]])
    assert np.max(np.abs(comp - np.eye(3))) < 1e-12
    # with noise: the linear least squares in (a, b, tx, ty) by numpy
    xn, yn = xt + rng.normal(0, 0.3, 500), yt + rng.normal(0, 0.3, 500)
    x[3], yn[7] = np.nan, np.inf
    M, _ = orc.affine_fit(x, y, xn, yn)
    ok = np.isfinite(x) & np.isfinite(yn)
    A = np.zeros((2 * ok.sum(), 4))
    A[0::2] = np.stack([x[ok], -y[ok], np.ones(ok.sum()), np.zeros(ok.sum())], 1)
    A[1::2] = np.stack([y[ok], x[ok], np.zeros(ok.sum()), np.ones(ok.sum())], 1)
    rhs = np.empty(2 * ok.sum()); rhs[0::2], rhs[1::2] = xn[ok], yn[ok]
    a, b, tx2, ty2 = np.linalg.lstsq(A, rhs, rcond=None)[0]
    assert np.max(np.abs(M - np.array([[a, -b, tx2], [b, a, ty2]]))) < 1e-8
    with pytest.raises(ValueError):
        orc.affine_fit([1.0, 1.0], [2.0, 2.0], [0.0, 0.0], [0.0, 0.0])


def test_reproject_translations_ramps_and_edges(orc):
    rng = np.random.default_rng(2)
    img = rng.normal(100, 10, (37, 53)).astype(np.float32)
    ident = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    assert np.array_equal(orc.reproject_affine(img, ident, 53, 37), img.astype(np.float64))
    # integer translation: out(j, i) = img(j + 3, i - 2); outside -> fill
    out = orc.reproject_affine(img, np.array([[1.0, 0, 3], [0, 1.0, -2]]), 53, 37, fill=-1.0)
    assert np.array_equal(out[2:, :50], img[:-2, 3:].astype(np.float64))
    assert np.all(out[:2] == -1.0) and np.all(out[:, 50:] == -1.0)
    # half-pixel shift: the mean of horizontal neighbours
    out = orc.reproject_affine(img, np.array([[1.0, 0, 0.5], [0, 1.0, 0]]), 52, 37)
    assert np.max(np.abs(out - (img[:, :-1].astype(np.float64) + img[:, 1:]) / 2)) < 1e-12
    # linear ramps are reproduced exactly by bilinear interpolation
    jj, ii = np.meshgrid(np.arange(64.0), np.arange(48.0))
    ramp = (3.0 + 0.25 * jj - 0.5 * ii).astype(np.float32)
    th = 0.2
    Mi = np.array([[0.9 * math.cos(th), -0.9 * math.sin(th), 10.0], [0.9 * math.sin(th), 0.9 * math.cos(th), 4.0]])
    out = orc.reproject_affine(ramp, Mi, 40, 40, fill=np.nan)
    xs = Mi[0, 0] * jj[:40, :40] + Mi[0, 1] * ii[:40, :40] + Mi[0, 2]
    ys = Mi[1, 0] * jj[:40, :40] + Mi[1, 1] * ii[:40, :40] + Mi[1, 2]
    inside = (xs >= 0) & (xs <= 63) & (ys >= 0) & (ys <= 47)
    assert inside.sum() > 800 and np.all(np.isnan(out[~inside]))
    assert np.max(np.abs(out[inside] - (3.0 + 0.25 * xs[inside] - 0.5 * ys[inside]))) < 1e-10
    # the last column is reachable; a hair beyond it is not; a NaN neighbour gives fill
    out = orc.reproject_affine(img, np.array([[0.0, 0, 52.0], [0, 1.0, 0]]), 1, 37)
    assert np.array_equal(out[:, 0], img[:, 52].astype(np.float64))
    out = orc.reproject_affine(img, np.array([[0.0, 0, 52.0 + 1e-9], [0, 1.0, 0]]), 1, 37, fill=7.0)
    assert np.all(out == 7.0)
    bad = img.copy(); bad[5, 5] = np.nan
    out = orc.reproject_affine(bad, np.array([[1.0, 0, 0.5], [0, 1.0, 0]]), 52, 37, fill=-3.0)
    assert out[5, 4] == -3.0 and out[5, 5] == -3.0 and np.isfinite(out[5, 6]) and np.isfinite(out[4, 4])

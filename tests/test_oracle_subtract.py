"""Pins of the oracle's image subtraction (Sec. 2.2.4, Eqs. 8-10; HOTPANTS-style
readings).  Each rests on something outside the oracle's formulas: a template
that is a single bright pixel returns the kernel itself, shifted (the
orientation of the convolution); a fixed kernel against scipy's convolve2d; the
tile-centre evaluation of a spatially varying kernel; exact recovery of a
kernel in the span of a small, well-conditioned basis and of the background
(noise-free synthetic pairs generated with scipy); with the full 49-function
basis the difference image vanishes and the kernel's sum (the photometric
scale) is recovered; stamp selection finds the stars."""
import math

import numpy as np
import pytest
from scipy.signal import convolve2d


def _stars(H, W, stars, sky=0.0):
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    img = np.full((H, W), sky)
    for x, y, F, s in stars:
        img += F / (2 * math.pi * s * s) * np.exp(-((j - x) ** 2 + (i - y) ** 2) / (2 * s * s))
    return img


def test_basis_layout_and_count(orc):
    B = orc.sub_basis(hw=10)
    assert B.shape == (49, 21, 21)               # 28 + 15 + 6 functions
    u = np.arange(-10, 11)
    # the first function of each Gaussian is the Gaussian itself, 1 at the centre
    for n, s in ((0, 0.7), (28, 1.5), (43, 3.0)):
        assert B[n, 10, 10] == 1.0
        assert np.allclose(B[n], np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * s * s)), rtol=1e-15, atol=0)
    # (i, j) = (0, 1) multiplies by v (rows), (1, 0) by u (columns): i outer, j inner
    g = B[0]
    assert np.allclose(B[1], g * u[:, None], rtol=1e-15, atol=0)
    assert np.allclose(B[7], g * u[None, :], rtol=1e-15, atol=0)   # i = 1, j = 0 follows the seven i = 0 terms


def test_single_pixel_template_returns_the_kernel(orc):
    """R = delta at (x0, y0): (R (x) K)(x, y) = K(x - x0, y - y0), so
    D = I - K(x - x0, y - y0) with I = 0, kernel constant (spatial order 0)."""
    H, W, hw = 40, 50, 4
    R = np.zeros((H, W), np.float32)
    R[20, 25] = 1.0
    I = np.zeros((H, W), np.float32)
    sig, deg = (1.0, 2.5), (2, 0)
    rng = np.random.default_rng(1)
    coef = rng.normal(0, 1, 7)       # 6 + 1 basis functions, no background
    D = orc.sub_apply(I, R, coef, hw=hw, sig=sig, deg=deg, sord=0, bord=-1, tile=9)
    K = np.tensordot(coef, orc.sub_basis(hw, sig, deg), 1)
    assert np.allclose(-D[20 - hw:21 + hw, 25 - hw:26 + hw], K, rtol=0, atol=1e-14)
    assert np.all(np.isnan(D[:hw])) and np.all(np.isnan(D[:, -hw:]))


def test_fixed_kernel_matches_convolve2d(orc):
    rng = np.random.default_rng(2)
    H, W, hw = 61, 73, 5
    R = rng.normal(100, 10, (H, W)).astype(np.float32)
    I = rng.normal(100, 10, (H, W)).astype(np.float32)
    sig, deg = (0.8, 2.0), (3, 1)
    coef = np.concatenate([rng.normal(0, 1, 13), [4.0, 0.5, -0.25]])   # 10 + 3 kernel, then 1, ys, xs
    D = orc.sub_apply(I, R, coef, hw=hw, sig=sig, deg=deg, sord=0, bord=1, tile=11)
    K = np.tensordot(coef[:13], orc.sub_basis(hw, sig, deg), 1)
    conv = convolve2d(R.astype(np.float64), K, mode="same")
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    xs, ys = 2 * j / (W - 1) - 1, 2 * i / (H - 1) - 1
    ref = I + (4.0 + 0.5 * ys - 0.25 * xs) - conv
    inner = (slice(hw, H - hw), slice(hw, W - hw))
    assert np.allclose(D[inner], ref[inner], rtol=0, atol=1e-9)


def test_kernel_taken_at_tile_centres(orc):
    """a_0(x, y) = 1 + 0.5 xs: pixels of one tile see one amplitude, the tile
    centre's"""
    H, W, hw, tile = 30, 60, 3, 7
    R = np.zeros((H, W), np.float32)
    I = np.zeros((H, W), np.float32)
    R[15, 10] = R[15, 40] = 1.0
    sig, deg = (1.0,), (0,)
    coef = np.array([1.0, 0.0, 0.5])            # terms 1, ys, xs
    D = orc.sub_apply(I, R, coef, hw=hw, sig=sig, deg=deg, sord=1, bord=-1, tile=tile)
    for x0 in (10, 40):
        for x in (x0 - 1, x0, x0 + 2):
            tcx = (x // tile) * tile + 0.5 * (tile - 1)
            amp = 1.0 + 0.5 * (2 * tcx / (W - 1) - 1)
            g = math.exp(-((x - x0) ** 2) / 2.0)
            assert -D[15, x] == pytest.approx(amp * g, rel=1e-13)


def _template(H=160, W=160):
    """noise-free template: 40 random stars and a bright star near the centre of
    each 40 px region"""
    rng = np.random.default_rng(7)
    stars = [(rng.uniform(20, W - 20), rng.uniform(20, H - 20), rng.uniform(2e3, 2e4), rng.uniform(1.0, 1.6))
             for _ in range(40)]
    stars += [(20 + 40 * a + 5.3, 20 + 40 * b + 3.7, 5e4, 1.3) for a in range(4) for b in range(4)]
    return _stars(H, W, stars, sky=100.0).astype(np.float32)


@pytest.mark.parametrize("bord", [-1, 1])
def test_exact_recovery_small_basis(orc, bord):
    H = W = 160
    hw = fh = 6
    sig, deg = (1.0, 2.5), (2, 0)
    R = _template()
    ck = np.array([0.6, 0.05, -0.02, 0.03, 0.01, -0.01, 0.02])
    K = np.tensordot(ck, orc.sub_basis(hw, sig, deg), 1)
    conv = convolve2d(R.astype(np.float64), K, mode="same")
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    xs, ys = 2 * j / (W - 1) - 1, 2 * i / (H - 1) - 1
    B = (5.0 - 3.0 * ys + 2.0 * xs) if bord == 1 else 0.0
    I = (conv - B).astype(np.float32)
    cx, cy = orc.sub_stamps(I, R, nsx=4, nsy=4, hw=hw, fh=fh, nsig=5.0)
    assert len(cx) == 16
    coef = orc.sub_fit(I, R, cx, cy, hw=hw, fh=fh, sig=sig, deg=deg, sord=0, bord=bord)
    # float32 rounding of I (~1e-7 relative) is the only error source
    assert np.allclose(coef[:7], ck, rtol=0, atol=2e-6)
    if bord == 1:
        assert np.allclose(coef[7:], [5.0, -3.0, 2.0], rtol=0, atol=2e-3)
    D = orc.sub_apply(I, R, coef, hw=hw, sig=sig, deg=deg, sord=0, bord=bord, tile=13)
    inner = (slice(hw, H - hw), slice(hw, W - hw))
    assert np.nanmax(np.abs(D[inner])) < 1e-4 * np.max(np.abs(conv))


def test_full_basis_scale_and_null_difference(orc):
    """the default 49-function basis and a kernel that is a normalised Gaussian
    of width 1.9 px (not in the span) times a flux ratio 0.8: the difference
    image is small against the stars and the fitted kernel's sum is the ratio"""
    H = W = 160
    hw = fh = 10
    R = _template()
    u = np.arange(-hw, hw + 1)
    G = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * 1.9 ** 2))
    K = 0.8 * G / G.sum()
    I = convolve2d(R.astype(np.float64), K, mode="same").astype(np.float32)
    cx, cy = orc.sub_stamps(I, R, nsx=4, nsy=4, hw=hw, fh=fh, nsig=5.0)
    coef = orc.sub_fit(I, R, cx, cy, hw=hw, fh=fh, sord=0, bord=0)
    Kfit = np.tensordot(coef[:49], orc.sub_basis(hw), 1)
    assert Kfit.sum() == pytest.approx(0.8, rel=1e-4)
    D = orc.sub_apply(I, R, coef, hw=hw, sord=0, bord=0, tile=21)
    inner = (slice(hw + 10, H - hw - 10), slice(hw + 10, W - hw - 10))
    assert np.nanmax(np.abs(D[inner])) < 1e-3 * np.max(I)


def test_stamp_selection(orc):
    H = W = 160
    R = _stars(H, W, [(20 + 40 * a + 5.3, 20 + 40 * b + 3.7, 5e4, 1.3) for a in range(4) for b in range(4)],
               sky=100.0)
    rng = np.random.default_rng(3)
    R = (R + rng.normal(0, 2.0, R.shape)).astype(np.float32)
    I = R.copy()
    R[120:, 120:] = 100.0                       # a flat region (3, 3): no candidate there
    I[62:66, 64:68] = np.nan                    # a NaN next to the star of region (1, 1)
    cx, cy = orc.sub_stamps(I, R, nsx=4, nsy=4, hw=6, fh=6, nsig=5.0)
    found = set(zip(cx.tolist(), cy.tolist()))
    expect = {(int(round(20 + 40 * a + 5.3)), int(round(20 + 40 * b + 3.7))) for a in range(4) for b in range(4)}
    # the flattened region gives nothing; next to the NaN the star's peak is not a
    # candidate (its footprint holds the NaN), a wing pixel of it may be
    assert not any(x >= 120 and y >= 120 for x, y in found)
    assert (65, 64) not in found
    assert len(found & expect) == 14 and len(found) <= 15


def test_normal_equations_match_an_explicit_design_matrix(orc):
    """the normal equations equal A'A and A'b of the design matrix built here from
    scipy convolutions of the template with each basis kernel, the spatial terms
    at the candidates' centres and the background terms at each pixel"""
    rng = np.random.default_rng(12)
    H, W, hw, fh = 70, 90, 4, 3
    R = (100 + rng.normal(0, 10, (H, W))).astype(np.float32)
    I = (100 + rng.normal(0, 10, (H, W))).astype(np.float32)
    sig, deg, sord, bord = (1.0, 2.0), (2, 1), 1, 1
    cx, cy = np.array([20, 55, 70], np.int32), np.array([15, 40, 50], np.int32)
    AtA, Atb = orc.sub_normal(I, R, cx, cy, hw=hw, fh=fh, sig=sig, deg=deg, sord=sord, bord=bord)
    B = orc.sub_basis(hw, sig, deg)
    conv = [convolve2d(R.astype(np.float64), B[n], mode="same") for n in range(B.shape[0])]

    def terms(x, y, order):
        xs, ys = 2.0 * x / (W - 1) - 1.0, 2.0 * y / (H - 1) - 1.0
        return [xs ** p * ys ** q for p in range(order + 1) for q in range(order + 1 - p)]

    rows, b = [], []
    for c in range(3):
        Ps = terms(cx[c], cy[c], sord)
        for dv in range(-fh, fh + 1):
            for du in range(-fh, fh + 1):
                x, y = cx[c] + du, cy[c] + dv
                r = [conv[n][y, x] * p for n in range(B.shape[0]) for p in Ps]
                r += [-t for t in terms(x, y, bord)]
                rows.append(r)
                b.append(float(I[y, x]))
    A, b = np.array(rows), np.array(b)
    assert AtA.shape == (A.shape[1], A.shape[1])
    assert np.allclose(AtA, A.T @ A, rtol=1e-11, atol=1e-6)
    assert np.allclose(Atb, A.T @ b, rtol=1e-11, atol=1e-6)
    # and the fit solves them
    coef = orc.sub_fit(I, R, cx, cy, hw=hw, fh=fh, sig=sig, deg=deg, sord=sord, bord=bord)
    assert np.allclose(coef, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-6, atol=1e-8)


def test_chol_solve_against_lapack(orc):
    """the oracle's Cholesky solve against LAPACK's (numpy) on a random SPD
    system, and a matrix with a zero pivot is refused"""
    rng = np.random.default_rng(12)
    M = rng.normal(0, 1, (40, 40))
    A = M @ M.T + 40 * np.eye(40)
    b = rng.normal(0, 1, 40)
    assert np.allclose(orc.chol_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-14)
    with pytest.raises(ValueError):
        orc.chol_solve(np.zeros((3, 3)), np.ones(3))

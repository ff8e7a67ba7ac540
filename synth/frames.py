"""Seeded star-field and stamp generators (numpy PCG64, ``default_rng(seed)``).

The fields stand in for the simulated survey images of the paper (Sec. 3.2,
SkyMaker fields shaped after the GWAC camera) and for its real GWAC frames
(4196 x 4136 px, ~20,000 sources; Sec. 3.3), neither of which is available.

Common recipe (all float frames):
  * pixel (row i, col j) has its centre at (x=j, y=i);
  * stars are rendered pixel-integrated: circular Gaussian products of
    normal-CDF differences over each pixel, truncated at 6 sigma;
  * Poisson noise on (sky + stars) with gain 1 e-/ADU, then N(0, 5^2) read noise;
  * draw order per frame: star positions, star fluxes, (widths), Poisson noise,
    read noise, then defects.

Nothing here estimates, detects or measures anything.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

FWHM_TO_SIGMA = 1.0 / (2.0 * np.sqrt(2.0 * np.log(2.0)))
READ_NOISE = 5.0


@dataclass
class FrameTruth:
    """Injected catalogue of a synthetic frame."""
    x: np.ndarray
    y: np.ndarray
    flux: np.ndarray
    fwhm: np.ndarray
    extra: dict = field(default_factory=dict)


def _phi(t):
    return 0.5 * (1.0 + erf(t / np.sqrt(2.0)))


def render_gaussian_stars(H, W, x, y, flux, sigma, chunk=4096):
    """Sum of pixel-integrated circular Gaussians, each truncated at 6 sigma.

    Returns a float64 H x W image of expected counts.
    """
    img = np.zeros(H * W, dtype=np.float64)
    n = len(x)
    if n == 0:
        return img.reshape(H, W)
    R = int(np.ceil(6.0 * float(np.max(sigma)))) + 1
    k = np.arange(-R, R + 1)
    for s in range(0, n, chunk):
        xs, ys = x[s:s + chunk], y[s:s + chunk]
        fs, ss = flux[s:s + chunk], sigma[s:s + chunk]
        jc = np.rint(xs).astype(np.int64)
        ic = np.rint(ys).astype(np.int64)
        jj = jc[:, None] + k[None, :]
        ii = ic[:, None] + k[None, :]
        ex = _phi((jj + 0.5 - xs[:, None]) / ss[:, None]) - _phi((jj - 0.5 - xs[:, None]) / ss[:, None])
        ey = _phi((ii + 0.5 - ys[:, None]) / ss[:, None]) - _phi((ii - 0.5 - ys[:, None]) / ss[:, None])
        ex = np.where(np.abs(jj - xs[:, None]) <= 6.0 * ss[:, None], ex, 0.0)
        ey = np.where(np.abs(ii - ys[:, None]) <= 6.0 * ss[:, None], ey, 0.0)
        ex = np.where((jj >= 0) & (jj < W), ex, 0.0)
        ey = np.where((ii >= 0) & (ii < H), ey, 0.0)
        val = fs[:, None, None] * ey[:, :, None] * ex[:, None, :]
        idx = np.clip(ii, 0, H - 1)[:, :, None] * W + np.clip(jj, 0, W - 1)[:, None, :]
        img += np.bincount(idx.ravel(), weights=val.ravel(), minlength=H * W)
    return img.reshape(H, W)


def _add_noise(rng, expected):
    counts = rng.poisson(np.maximum(expected, 0.0)).astype(np.float64)
    return counts + rng.normal(0.0, READ_NOISE, size=expected.shape)


def _normalised_coords(H, W):
    xh = 2.0 * np.arange(W, dtype=np.float64) / max(W - 1, 1) - 1.0
    yh = 2.0 * np.arange(H, dtype=np.float64) / max(H - 1, 1) - 1.0
    return xh, yh


def frame_field(W, H, n_stars, seed, sky_level=1000.0, grad=50.0, fwhm=3.0,
                logflux=(2.5, 5.0)):
    """Generic field: sky + linear x gradient of +-grad ADU, uniform positions,
    log-uniform fluxes 10^(a + (b-a) u), fixed FWHM, Poisson + read noise."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, W, n_stars)
    y = rng.uniform(0.0, H, n_stars)
    a, b = logflux
    flux = 10.0 ** (a + (b - a) * rng.uniform(0.0, 1.0, n_stars))
    sig = np.full(n_stars, fwhm * FWHM_TO_SIGMA)
    xh, _ = _normalised_coords(H, W)
    sky = sky_level + grad * np.broadcast_to(xh[None, :], (H, W))
    expected = sky + render_gaussian_stars(H, W, x, y, flux, sig)
    img = _add_noise(rng, expected).astype(np.float32)
    return img, FrameTruth(x, y, flux, np.full(n_stars, fwhm), {"sky": sky})


def frame_gradient_1k(seed=1001):
    """1024 x 1024 field: sky 1000 ADU with a +-50 ADU gradient along x,
    500 stars of FWHM 3 px, fluxes 10^2.5 .. 10^5 ADU log-uniform."""
    return frame_field(1024, 1024, 500, seed)


def frame_survey_4k(seed=1002, W=4096, H=4096, n_stars=20000):
    """4096 x 4096 survey-like field.

    sky = 1000 + 200 (xh^2 + yh^2 - 1) (800..1200 ADU), 20,000 stars with FWHM
    rising linearly from 2.5 px (x=0) to 4 px (x=W-1), power-law fluxes
    dN/dF ~ F^-1.5 on [1e2, 1e6], then 0.01% hot pixels set to sky + 5e4 ADU and
    200 cosmic-ray tracks (1-px DDA lines, length U[1,10] px, random angle,
    +1e4 ADU per pixel).
    """
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, W, n_stars)
    y = rng.uniform(0.0, H, n_stars)
    a, b = 1e2 ** -0.5, 1e6 ** -0.5
    flux = (a - rng.uniform(0.0, 1.0, n_stars) * (a - b)) ** -2.0
    fwhm = 2.5 + 1.5 * x / (W - 1)
    xh, yh = _normalised_coords(H, W)
    sky = 1000.0 + 200.0 * (xh[None, :] ** 2 + yh[:, None] ** 2 - 1.0)
    expected = sky + render_gaussian_stars(H, W, x, y, flux, fwhm * FWHM_TO_SIGMA)
    img = _add_noise(rng, expected)
    n_hot = int(round(1e-4 * W * H))
    hot = rng.choice(W * H, size=n_hot, replace=False)
    img.ravel()[hot] = sky.ravel()[hot] + 5e4
    cr_pix = []
    for _ in range(200):
        x0, y0 = rng.uniform(0.0, W), rng.uniform(0.0, H)
        L = rng.uniform(1.0, 10.0)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        c, s = np.cos(ang), np.sin(ang)
        m = max(abs(c), abs(s))
        n = int(np.ceil(L * m)) + 1
        t = np.arange(n)
        cj = np.rint(x0 + t * c / m).astype(np.int64)
        ci = np.rint(y0 + t * s / m).astype(np.int64)
        ok = (cj >= 0) & (cj < W) & (ci >= 0) & (ci < H)
        pix = np.unique(ci[ok] * W + cj[ok])
        img.ravel()[pix] += 1e4
        cr_pix.append(pix)
    truth = FrameTruth(x, y, flux, fwhm, {"sky": sky, "hot": hot, "cosmic": cr_pix})
    return img.astype(np.float32), truth


def frame_field_device(W, H, n_stars, seed, sky_level=1000.0, grad=50.0, fwhm=3.0, logflux=(2.5, 5.0),
                       device="cuda"):
    """The frame_field recipe drawn with a seeded torch generator on the device
    (for the large batches of the benchmark, where the host generator would
    take minutes): uniform positions, log-uniform fluxes, pixel-integrated
    Gaussians truncated at 6 sigma, linear x gradient, Poisson + read noise.
    Returns a float32 H x W tensor on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    x = torch.rand(n_stars, generator=g, device=device, dtype=f64) * W
    y = torch.rand(n_stars, generator=g, device=device, dtype=f64) * H
    a, b = logflux
    flux = 10.0 ** (a + (b - a) * torch.rand(n_stars, generator=g, device=device, dtype=f64))
    sig = fwhm * FWHM_TO_SIGMA
    xh = 2.0 * torch.arange(W, device=device, dtype=f64) / max(W - 1, 1) - 1.0
    expected = (sky_level + grad * xh)[None, :].expand(H, W).reshape(-1).clone()
    R = int(np.ceil(6.0 * sig)) + 1
    k = torch.arange(-R, R + 1, device=device, dtype=torch.int64)
    phi = lambda t: 0.5 * (1.0 + torch.special.erf(t / np.sqrt(2.0)))
    for s0 in range(0, n_stars, 8192):
        xs, ys, fs = x[s0:s0 + 8192], y[s0:s0 + 8192], flux[s0:s0 + 8192]
        jj = torch.round(xs).long()[:, None] + k[None, :]
        ii = torch.round(ys).long()[:, None] + k[None, :]
        ex = phi((jj + 0.5 - xs[:, None]) / sig) - phi((jj - 0.5 - xs[:, None]) / sig)
        ey = phi((ii + 0.5 - ys[:, None]) / sig) - phi((ii - 0.5 - ys[:, None]) / sig)
        ex = torch.where(((jj - xs[:, None]).abs() <= 6 * sig) & (jj >= 0) & (jj < W), ex, 0.0)
        ey = torch.where(((ii - ys[:, None]).abs() <= 6 * sig) & (ii >= 0) & (ii < H), ey, 0.0)
        val = fs[:, None, None] * ey[:, :, None] * ex[:, None, :]
        idx = ii.clamp(0, H - 1)[:, :, None] * W + jj.clamp(0, W - 1)[:, None, :]
        expected.index_add_(0, idx.reshape(-1), val.reshape(-1))
    counts = torch.poisson(expected.clamp_min(0.0), generator=g)
    img = counts + READ_NOISE * torch.randn(counts.shape, generator=g, device=device, dtype=f64)
    return img.reshape(H, W).float()


def mixed_batch_shapes(n_frames=64):
    """Frame shapes (W, H) of the mixed batch: 2048^2, 4096^2, 6144 x 6160 by i mod 3."""
    table = [(2048, 2048), (4096, 4096), (6144, 6160)]
    return [table[i % 3] for i in range(n_frames)]


def raw_calibrated_4k(seed=5000, W=4096, H=4096, n_stars=8000, bias=500.0):
    """Raw uint16 frame with bias 500 ADU and a radial flat 1.1 - 0.2 (r/r_max)^2.

    raw = clip(round(bias + flat * (scene + noise)), 0, 65535); the scene is the
    1k-field recipe at 4096^2 (same star density).  Returns (raw, flat, truth).
    """
    img, truth = frame_field(W, H, n_stars, seed)
    yy, xx = np.mgrid[0:H, 0:W]
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    r = np.hypot(xx - cx, yy - cy)
    flat = (1.1 - 0.2 * (r / r.max()) ** 2).astype(np.float32)
    raw = np.clip(np.rint(bias + flat.astype(np.float64) * img), 0, 65535).astype(np.uint16)
    return raw, flat, truth


def moffat_stamps(n, seed=4000, S=15, beta=2.5, oversample=5):
    """n elliptical Moffat stamps of S x S px with Poisson + read noise.

    Truth per stamp: x, y = 7 + U(-0.5, 0.5); flux from the F^-1.5 power law on
    [1e2, 1e6]; sky U[800, 1200]; core widths ax, ay ~ U[1, 2] px; angle U[0, pi).
    The profile F (beta-1)/(pi ax ay) (1 + u^2/ax^2 + v^2/ay^2)^-beta is
    integrated over each pixel by averaging oversample^2 sub-pixel samples.
    Returns (stamps float32 [n, S, S], truth float64 [n, 7]).
    """
    rng = np.random.default_rng(seed)
    c = (S - 1) / 2.0
    x0 = c + rng.uniform(-0.5, 0.5, n)
    y0 = c + rng.uniform(-0.5, 0.5, n)
    a, b = 1e2 ** -0.5, 1e6 ** -0.5
    flux = (a - rng.uniform(0.0, 1.0, n) * (a - b)) ** -2.0
    sky = rng.uniform(800.0, 1200.0, n)
    ax = rng.uniform(1.0, 2.0, n)
    ay = rng.uniform(1.0, 2.0, n)
    th = rng.uniform(0.0, np.pi, n)
    off = (np.arange(oversample) + 0.5) / oversample - 0.5
    px = np.arange(S, dtype=np.float64)
    sub = (px[:, None] + off[None, :]).ravel()  # S*os sample coordinates
    out = np.empty((n, S, S), dtype=np.float32)
    chunk = 2048
    for s in range(0, n, chunk):
        e = slice(s, min(n, s + chunk))
        dx = sub[None, None, :] - x0[e, None, None]
        dy = sub[None, :, None] - y0[e, None, None]
        ct, st = np.cos(th[e])[:, None, None], np.sin(th[e])[:, None, None]
        u = ct * dx + st * dy
        v = -st * dx + ct * dy
        q = (u / ax[e, None, None]) ** 2 + (v / ay[e, None, None]) ** 2
        norm = flux[e] * (beta - 1.0) / (np.pi * ax[e] * ay[e])
        prof = norm[:, None, None] * (1.0 + q) ** (-beta)
        m = len(range(*e.indices(n)))
        prof = prof.reshape(m, S, oversample, S, oversample).mean(axis=(2, 4))
        expected = prof + sky[e, None, None]
        out[e] = _add_noise(rng, expected).astype(np.float32)
    truth = np.stack([x0, y0, flux, sky, ax, ay, th], axis=1)
    return out, truth


def tiny_frame(W, H, seed, n_stars=4, sky=100.0, fwhm=2.5, flux=(3.0, 4.0)):
    """Small field for parity tests that must span several tiles with a ragged tail."""
    return frame_field(W, H, n_stars, seed, sky_level=sky, grad=10.0, fwhm=fwhm, logflux=flux)


def wcs_pair(W=4096, H=4096, seed=7000, scale_arcsec=1.5, order=3):
    """Headers of two overlapping exposures of one field, as a survey camera
    with a few pixels of optical distortion at the corners would carry them:
    a source and a target WCS (dicts: crpix, crval, cd, a, b, a_order,
    b_order).  The target is pointed 0.02-0.05 degrees away, rotated by up to
    half a degree, with its own distortion.  Header values only; no mapping."""
    rng = np.random.default_rng(seed)
    s = scale_arcsec / 3600.0

    def one(ra, dec, rot, k):
        c, sn = np.cos(rot), np.sin(rot)
        a, b = np.zeros((6, 6)), np.zeros((6, 6))
        half = max(W, H) / 2.0
        for p in range(6):
            for q in range(6 - p):
                if 2 <= p + q <= order:
                    a[p, q] = rng.normal(0.0, 1.0) * 2.0 * half ** (-p - q)
                    b[p, q] = rng.normal(0.0, 1.0) * 2.0 * half ** (-p - q)
        return dict(crpix=[W / 2.0 + 0.5 + k, H / 2.0 + 0.5 - k], crval=[ra, dec],
                    cd=[[-s * c, s * sn], [s * sn, s * c]], a=a, b=b, a_order=order, b_order=order)

    ra0, dec0 = rng.uniform(0.0, 360.0), rng.uniform(-60.0, 60.0)
    src = one(ra0, dec0, rng.uniform(-0.01, 0.01), 0.0)
    tgt = one(ra0 + rng.uniform(0.02, 0.05) / np.cos(np.radians(dec0)), dec0 + rng.uniform(-0.05, -0.02),
              rng.uniform(0.2, 0.5) * np.pi / 180.0, 3.25)
    return src, tgt

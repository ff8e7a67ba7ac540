"""GPU parity of image alignment (Sec. 2.2.3) with the oracle.

Mapping: both sides in FP64, the GPU composing Eq. 7 and the target's gnomonic
projection as one rotation (no trigonometric call per node) and the oracle with
Eq. 7's trigonometry: the target positions agree to 1e-7 px (the rounding of a
few dozen FP64 operations on coordinates of a few thousand px, 1e-12 px, times
the conditioning of Newton's inverse; a wide margin).  NaN where the oracle has
NaN.

Affine fit: FP64 sums in different orders: 1e-12 relative on M.

Reprojection: the GPU position is formed in FP64 once per 128 output pixels and
offset in FP32, within 2e-5 px of the FP64 position; the bilinear sum is FP32.
So |gpu - oracle| <= 4e-5 (max - min of the four neighbours) + 1e-6 max|neighbour|.
Pixels whose FP64 position lies within 1e-4 px of the edge of the defined region
(where the two sides may take the inside/outside decision differently) are left
out of the comparison; every other fill decision must match."""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _grid(W, H, step):
    return np.meshgrid(np.arange(0, W, step, dtype=np.float64), np.arange(0, H, step, dtype=np.float64))


def _reproject_check(orc, img, Mi, Wo, Ho, g, fill):
    """compare a GPU reprojection with the oracle's, away from the region's edge"""
    H, W = img.shape
    o = orc.reproject_affine(img, Mi, Wo, Ho, fill=fill)
    jj, ii = np.meshgrid(np.arange(Wo, dtype=np.float64), np.arange(Ho, dtype=np.float64))
    x = Mi[0, 0] * jj + Mi[0, 1] * ii + Mi[0, 2]
    y = Mi[1, 0] * jj + Mi[1, 1] * ii + Mi[1, 2]
    e = 1e-4
    near = ((np.abs(x) < e) | (np.abs(x - (W - 1)) < e) | (np.abs(y) < e) | (np.abs(y - (H - 1)) < e))
    inside = (x >= 0) & (x <= W - 1) & (y >= 0) & (y <= H - 1) & ~near
    outside = ~inside & ~near
    f = img.astype(np.float64)
    bad_src = ~np.isfinite(f)
    if np.isnan(fill):
        assert np.all(np.isnan(g[outside]))
    else:
        assert np.all(g[outside] == np.float32(fill))
    x0 = np.clip(np.floor(x[inside]).astype(np.int64), 0, max(W - 2, 0))
    y0 = np.clip(np.floor(y[inside]).astype(np.int64), 0, max(H - 2, 0))
    x1, y1 = np.minimum(x0 + 1, W - 1), np.minimum(y0 + 1, H - 1)
    nb = np.stack([f[y0, x0], f[y0, x1], f[y1, x0], f[y1, x1]])
    has_bad = bad_src[y0, x0] | bad_src[y0, x1] | bad_src[y1, x0] | bad_src[y1, x1]
    ok = ~has_bad   # a non-finite neighbour with zero weight is not read: compare those pixels by fill below
    span = np.nanmax(nb, 0) - np.nanmin(nb, 0)
    tol = 4e-5 * span + 1e-6 * np.nanmax(np.abs(nb), 0)
    gi, oi = g[inside], o[inside]
    assert np.all(np.abs(gi[ok] - oi[ok]) <= tol[ok] + 1e-30)
    # pixels with a non-finite neighbour: both give fill, or both the same finite value
    both = has_bad
    if both.any():
        same_fill = (np.isnan(gi[both]) & np.isnan(oi[both])) if np.isnan(fill) else (gi[both] == oi[both])
        fin = np.isfinite(oi[both]) & np.isfinite(gi[both])
        assert np.all(same_fill | (fin & (np.abs(gi[both] - oi[both]) <= 1e-3 * (1 + np.abs(oi[both])))))
    return int(inside.sum())


@pytest.mark.parametrize("W,H,step", [(4096, 4096, 64), (517, 389, 1), (1001, 77, 7)])
def test_wcs_map_parity(gpu, orc, W, H, step):
    src, tgt = synth.wcs_pair(W, H, seed=7000 + step)
    gx, gy = gpu.wcs_map(src, tgt, W, H, step=step)
    ox, oy = orc.wcs_map(src, tgt, W, H, step=step)
    gx, gy = host(gx), host(gy)
    assert gx.shape == ox.shape
    assert np.array_equal(np.isnan(gx), np.isnan(ox))
    assert np.nanmax(np.abs(gx - ox)) <= 1e-7 and np.nanmax(np.abs(gy - oy)) <= 1e-7


def test_wcs_map_edge_cases(gpu, orc):
    src, tgt = synth.wcs_pair(300, 200, seed=7100)
    # identical frames: the identity
    gx, gy = gpu.wcs_map(src, src, 300, 200, step=13)
    X, Y = _grid(300, 200, 13)
    assert np.max(np.abs(host(gx) - X)) < 1e-8 and np.max(np.abs(host(gy) - Y)) < 1e-8
    # a target pointed at the antipode: no point has an image
    far = dict(tgt, crval=[tgt["crval"][0] + 180.0, -tgt["crval"][1]])
    gx, _ = gpu.wcs_map(src, far, 300, 200, step=50)
    ox, _ = orc.wcs_map(src, far, 300, 200, step=50)
    assert np.all(np.isnan(host(gx))) and np.all(np.isnan(ox))
    # one pixel
    gx, gy = gpu.wcs_map(src, tgt, 1, 1, step=1)
    ox, oy = orc.wcs_map(src, tgt, 1, 1, step=1)
    assert abs(host(gx)[0, 0] - ox[0, 0]) < 1e-7 and abs(host(gy)[0, 0] - oy[0, 0]) < 1e-7
    with pytest.raises(gpu.IppError):
        gpu.wcs_map(dict(src, a_order=6), tgt, 10, 10)
    with pytest.raises(gpu.IppError):
        gpu.wcs_map(src, dict(tgt, cd=[[2.0 ** -12, 2.0 ** -13], [2.0 ** -11, 2.0 ** -12]]), 10, 10)


def test_affine_fit_parity(gpu, orc):
    src, tgt = synth.wcs_pair(4096, 4096, seed=7200)
    xo, yo = orc.wcs_map(src, tgt, 4096, 4096, step=32)
    X, Y = _grid(4096, 4096, 32)
    xo[3, 4] = np.nan   # a node without an image is skipped
    Mo, Mio = orc.affine_fit(X, Y, xo, yo)
    Mg, st = gpu.affine_fit(dev(xo), dev(yo), grid_step=32)
    Mg = host(Mg)
    assert int(host(st)[0]) == 0
    ref = np.concatenate([Mo.ravel(), Mio.ravel()])
    assert np.max(np.abs(Mg - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
    # explicit point lists give the same answer
    Mg2, _ = gpu.affine_fit(dev(xo.ravel()), dev(yo.ravel()), x=dev(X.ravel()), y=dev(Y.ravel()))
    assert np.max(np.abs(host(Mg2) - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
    # degenerate: no usable pair, one pair, coincident pairs
    nan = np.full(10, np.nan)
    for xs, ys in ((nan, nan), (np.array([1.0]), np.array([2.0]))):
        M, st = gpu.affine_fit(dev(xs), dev(ys), x=dev(np.zeros_like(xs)), y=dev(np.zeros_like(xs)))
        assert int(host(st)[0]) == gpu._abi.IPP_ERR_DEGENERATE and np.all(np.isnan(host(M)))
    M, st = gpu.affine_fit(dev(np.ones(4)), dev(np.ones(4)), x=dev(np.full(4, 2.0)), y=dev(np.full(4, 3.0)))
    assert int(host(st)[0]) == gpu._abi.IPP_ERR_DEGENERATE


@pytest.mark.parametrize("case", ["rotation", "ragged_views", "nan_fill"])
def test_reproject_parity(gpu, orc, case):
    img, _ = synth.tiny_frame(517, 389, 91, n_stars=50, sky=300.0, flux=(3.0, 4.5))
    th, s = 0.6 * math.pi / 180.0, 1.0003
    Mi = np.array([[s * math.cos(th), -s * math.sin(th), 3.3], [s * math.sin(th), s * math.cos(th), -2.7]])
    fill = 0.0
    if case == "ragged_views":
        big = dev(img)
        srcv = big[:, 1:]                                # unaligned base, pitch 517
        img = img[:, 1:]
        out = torch.full((420, 600), -9.0, device="cuda")
        g = gpu.reproject_affine(srcv, dev(Mi.ravel()), 530, 401, fill=fill, out=out[:401, :530])
        assert torch.all(out[:, 530:] == -9.0) and torch.all(out[401:] == -9.0)
        n = _reproject_check(orc, img, Mi, 530, 401, host(g), fill)
    else:
        if case == "nan_fill":
            img = img.copy()
            img[100:103, 200:240] = np.nan
            fill = float("nan")
        g = gpu.reproject_affine(dev(img), dev(Mi.ravel()), 530, 401, fill=fill)
        n = _reproject_check(orc, img, Mi, 530, 401, host(g), fill)
    assert n > 150000


def test_reproject_exact_cases(gpu):
    rng = np.random.default_rng(4)
    img = rng.normal(100, 10, (61, 75)).astype(np.float32)
    d = dev(img)
    ident = dev(np.array([1.0, 0, 0, 0, 1.0, 0]))
    assert np.array_equal(host(gpu.reproject_affine(d, ident, 75, 61)), img)
    g = host(gpu.reproject_affine(d, dev(np.array([1.0, 0, 3, 0, 1.0, -2])), 75, 61, fill=-1.0))
    assert np.array_equal(g[2:, :72], img[:-2, 3:]) and np.all(g[:2] == -1.0) and np.all(g[:, 72:] == -1.0)
    # the last column is defined; just beyond it is not
    g = host(gpu.reproject_affine(d, dev(np.array([0.0, 0, 74.0, 0, 1.0, 0])), 1, 61, fill=5.0))
    assert np.array_equal(g[:, 0], img[:, 74])
    g = host(gpu.reproject_affine(d, dev(np.array([0.0, 0, 74.001, 0, 1.0, 0])), 1, 61, fill=5.0))
    assert np.all(g == 5.0)
    # a NaN transform maps nothing
    g = host(gpu.reproject_affine(d, dev(np.full(6, np.nan)), 8, 8, fill=2.0))
    assert np.all(g == 2.0)
    with pytest.raises(gpu.IppError):
        gpu.reproject_affine(d, ident, 75, 61, out=d)


@pytest.mark.parametrize("which", ["survey_4k"])
def test_align_chain_full_size(gpu, orc, which):
    """map (step 32) -> fit -> reproject on the 4096^2 survey frame, against the
    oracle's chain on the same inputs; every output pixel compared"""
    img, _ = synth.frame_survey_4k()
    src, tgt = synth.wcs_pair(4096, 4096, seed=7300)
    out, M, st = gpu.align(dev(img), src, tgt, 4096, 4096, step=32, fill=0.0)
    assert int(host(st)[0]) == 0
    xo, yo = orc.wcs_map(src, tgt, 4096, 4096, step=32)
    X, Y = _grid(4096, 4096, 32)
    Mo, Mio = orc.affine_fit(X, Y, xo, yo)
    ref = np.concatenate([Mo.ravel(), Mio.ravel()])
    Mg = host(M)
    assert np.max(np.abs(Mg - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-11
    n = _reproject_check(orc, img, Mg[6:].reshape(2, 3), 4096, 4096, host(out), 0.0)
    assert n > 15_000_000


def test_reproject_full_8k(gpu, orc):
    """the 8192^2 maximum case (256 MiB, above L2) through a rotation and scale,
    every output pixel compared"""
    from test_gpu_gray import _big_frame
    img = _big_frame()
    th, s = 0.3 * math.pi / 180.0, 0.9995
    Mi = np.array([[s * math.cos(th), -s * math.sin(th), 20.5], [s * math.sin(th), s * math.cos(th), -11.25]])
    g = gpu.reproject_affine(dev(img), dev(Mi.ravel()), 8192, 8192, fill=0.0)
    assert _reproject_check(orc, img, Mi, 8192, 8192, host(g), 0.0) > 60_000_000

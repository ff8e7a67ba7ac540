"""Pins of the oracle's background steps (Sec. 2.2.2, Eqs. 1-4) to values that
do not come from the oracle itself: hand-worked golden cases, closed forms,
library routines and invariants."""
import json
import os

import numpy as np
import pytest
from scipy import ndimage, optimize, stats

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _one_mesh(values):
    v = np.asarray(values, dtype=np.float32)
    return v.reshape(1, -1)


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "mesh_clip_cases.json")))["cases"],
                         ids=lambda c: c["name"])
def test_clip_golden(orc, case):
    img = _one_mesh(case["values"])
    n = img.shape[1]
    st = orc.mesh_stats(img, mesh=n, mesh_h=1, min_valid=1, estimator=case["estimator"],
                        median_factor=case.get("median_factor", 2.5),
                        mean_factor=case.get("mean_factor", 1.5))
    assert st["valid"][0, 0] == 1
    assert st["raw_bkg"][0, 0] == pytest.approx(case["bkg"], abs=1e-12)
    assert st["raw_rms"][0, 0] == pytest.approx(case["rms"], rel=1e-12)
    assert st["niter"][0, 0] == case["passes"]


def test_constant_mesh_exact(orc):
    img = np.full((128, 192), 1234.5625, np.float32)
    st = orc.mesh_stats(img, mesh=64)
    assert np.all(st["raw_bkg"] == 1234.5625)
    assert np.all(st["raw_rms"] == 0.0)
    bkg, rms, _ = orc.bg_estimate(img, mesh=64)
    assert np.all(bkg == np.float32(1234.5625)) and np.all(rms == 0)


def test_gaussian_clip_fixed_point(orc):
    """Large Gaussian sample: the clipped sigma converges to c*sigma where c is
    the fixed point of 'std of N(0,1) truncated at +-3c equals c' (truncated-
    normal variance 1 - 2a phi(a)/(2 Phi(a) - 1) at a = 3c); the mode estimator
    of a symmetric distribution is its centre."""
    rng = np.random.default_rng(7)
    mu, sig = 500.0, 20.0
    img = (mu + sig * rng.standard_normal((1000, 1000))).astype(np.float32)

    def g(c):
        a = 3.0 * c
        var = 1.0 - 2.0 * a * stats.norm.pdf(a) / (2.0 * stats.norm.cdf(a) - 1.0)
        return np.sqrt(var) - c
    c = optimize.brentq(g, 0.9, 1.0)
    assert 0.98 < c < 0.99
    st = orc.mesh_stats(img, mesh=1000, maxiters=50)
    assert st["raw_bkg"][0, 0] == pytest.approx(mu, abs=6 * sig / 1000)
    assert st["raw_rms"][0, 0] == pytest.approx(c * sig, rel=4e-3)


def test_partial_and_masked_meshes(orc):
    """Partial last meshes keep their real pixels; masked pixels are excluded;
    meshes with fewer than 100 usable pixels are invalid (Sec. 2.2.2)."""
    rng = np.random.default_rng(3)
    img = (100 + rng.standard_normal((70, 130))).astype(np.float32)
    img[:, 128:] = 7.0          # the 2-px-wide last mesh column holds only 7s
    mask = np.zeros(img.shape, np.uint8)
    mask[0:64, 0:64] = 1        # fully masked mesh -> invalid
    mask[64:70, 64:128] = 1     # partial bottom mesh (6 rows) fully masked -> invalid
    st = orc.mesh_stats(img, mask=mask, mesh=64)
    assert st["valid"].shape == (2, 3)
    assert st["valid"][0, 0] == 0 and st["valid"][1, 1] == 0
    assert st["valid"][0, 2] == 1 and st["raw_bkg"][0, 2] == 7.0   # 2x64 = 128 px >= 100
    assert st["valid"][1, 2] == 0                                   # 2x6 = 12 px < 100
    assert st["valid"][1, 0] == 1                                   # 64x6 = 384 px >= 100
    assert st["valid"][0, 1] == 1


def test_partial_mesh_valid_counts(orc):
    rng = np.random.default_rng(3)
    img = (100 + rng.standard_normal((70, 130))).astype(np.float32)
    st = orc.mesh_stats(img, mesh=64)
    # rows 64..69 give 6-row meshes: 6*64 = 384 px valid, 6*2 = 12 px invalid
    assert st["valid"].tolist() == [[1, 1, 1], [1, 1, 0]]
    # the value of a partial mesh uses exactly its own pixels
    sub = img[64:70, 0:64].astype(np.float64)
    one = orc.mesh_stats(np.ascontiguousarray(img[64:70, 0:64]), mesh=64)
    assert st["raw_bkg"][1, 0] == one["raw_bkg"][0, 0]
    assert np.isfinite(sub).all()


def test_median_filter_golden(orc):
    g = json.load(open(os.path.join(GOLD, "mesh_filter_4x4.json")))
    grid = np.array(g["grid"], float)
    valid = np.ones(grid.shape, np.int32)
    b, r = orc.fill_filter(grid, grid / 10, valid, 3)
    assert np.array_equal(b, np.array(g["filtered"]))
    assert np.allclose(r, np.array(g["filtered"]) / 10, rtol=0, atol=1e-15)
    fc = g["fill_case"]
    grid = np.array(fc["grid"], float)
    valid = np.ones(grid.shape, np.int32)
    for (p, q) in fc["invalid"]:
        valid[p, q] = 0
    b, _ = orc.fill_filter(grid, grid / 10, valid, 1)   # filter of size 1 = fill only
    assert b[1, 1] == fc["filled_value"]
    assert np.array_equal(np.delete(b.ravel(), 5), np.delete(grid.ravel(), 5))


def test_median_filter_vs_scipy(orc):
    """Shrinking-window median == scipy generic_filter over NaN-padded input
    with numpy's nanmedian (even counts average the two middle values)."""
    rng = np.random.default_rng(11)
    for shape in [(1, 1), (1, 5), (4, 7), (9, 6)]:
        grid = rng.normal(size=shape)
        b, _ = orc.fill_filter(grid, grid, np.ones(shape, np.int32), 3)
        ref = ndimage.generic_filter(grid, np.nanmedian, size=3, mode="constant", cval=np.nan)
        assert np.allclose(b, ref, rtol=0, atol=1e-14)
    with pytest.raises(ValueError):
        orc.fill_filter(np.zeros((2, 2)), np.zeros((2, 2)), np.zeros((2, 2), np.int32), 3)


def test_keys_kernel_golden(orc):
    g = json.load(open(os.path.join(GOLD, "keys_kernel.json")))
    for s, w in g["points"]:
        assert orc.keys_weight(s) == pytest.approx(w, abs=1e-15)
    for s in np.linspace(0, 1, 37):
        tot = sum(orc.keys_weight(s - k) for k in (-1, 0, 1, 2))
        assert tot == pytest.approx(1.0, abs=1e-14)


def test_interp_constant_and_quadratic(orc):
    """Keys a=-1/2 reproduces polynomials up to degree 2 exactly where the 4x4
    node support is in bounds; a constant grid is reproduced exactly everywhere."""
    B, nx, ny = 8, 9, 7
    W, H = nx * B, ny * B
    const = np.full((ny, nx), 321.25, np.float32)
    m = orc.interp_map(const, B, W, H)
    assert np.all(m == 321.25)
    qx = (np.arange(nx) + 0.5) * B - 0.5
    qy = (np.arange(ny) + 0.5) * B - 0.5

    def f(x, y):
        return 3.0 + 0.25 * x - 0.5 * y + 0.01 * x * x - 0.02 * x * y + 0.005 * y * y
    nodes = f(qx[None, :], qy[:, None]).astype(np.float32)
    fexact = f(qx[None, :].astype(np.float64), qy[:, None]).astype(np.float32).astype(np.float64)
    m = orc.interp_map(nodes, B, W, H)
    # interior: pixel (i,j) whose lower node index q0 satisfies 1 <= q0 <= nx-3
    jj = np.arange(W)
    ii = np.arange(H)
    q0 = np.floor((jj + 0.5) / B - 0.5).astype(int)
    p0 = np.floor((ii + 0.5) / B - 0.5).astype(int)
    okx = (q0 >= 1) & (q0 <= nx - 3)
    oky = (p0 >= 1) & (p0 <= ny - 3)
    # node values are float32-rounded; compare with the quadratic through those
    # rounded values only up to their rounding (|f| < 20 -> 2e-6)
    want = f(jj[None, :].astype(float), ii[:, None].astype(float))
    err = np.abs(m - want)[np.ix_(oky, okx)]
    assert np.max(np.abs(nodes - fexact)) < 2e-6
    assert err.max() < 1e-5
    assert np.all(np.isfinite(m))


def test_interp_node_centres_exact(orc):
    """With odd mesh size the node sits on a pixel centre: B there equals the node."""
    B, nx, ny = 5, 6, 4
    rng = np.random.default_rng(5)
    nodes = rng.uniform(10, 20, (ny, nx)).astype(np.float32)
    m = orc.interp_map(nodes, B, nx * B, ny * B)
    for p in range(ny):
        for q in range(nx):
            assert m[p * B + 2, q * B + 2] == pytest.approx(float(nodes[p, q]), abs=1e-12)


def test_subtract_constant_sky_zero_residual(orc):
    img = np.full((200, 330), 987.375, np.float32)
    bkg, rms, _ = orc.bg_estimate(img, mesh=64)
    sub, bmap = orc.bg_subtract(img, bkg, 64)
    assert np.all(sub == 0.0) and np.all(bmap == np.float32(987.375))
    m = orc.threshold(sub, rms, 64, 1.5)
    assert m.sum() == 0


def test_gradient_sky_recovered(orc):
    """A noise-free linear sky is recovered exactly away from the frame edges
    (median of a linear ramp = its mean = its value at the mesh centre)."""
    H, W, B = 256, 384, 32
    yy, xx = np.mgrid[0:H, 0:W]
    sky = (1000.0 + 0.5 * xx - 0.25 * yy).astype(np.float32)
    bkg, rms, st = orc.bg_estimate(sky, mesh=B, filter_size=1)
    sub, _ = orc.bg_subtract(sky, bkg, B)
    inner = sub[2 * B:-2 * B, 2 * B:-2 * B]
    assert np.abs(inner).max() < 1e-3

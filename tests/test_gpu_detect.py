"""GPU parity of detection and labeling (Sec. 2.2.5): given the same mask the
label map, the count and the integer statistics are bit-exact against the
oracle's raster-order flood fill; flux sums within 1e-5 relative; barycentres
within 2 float32 ulps + 2e-5 px.  Masks span several 32 x 128 tiles with ragged
edges, and include the degenerate cases of the method."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, float_ulp, host, pack_mask, rel_close

pytestmark = pytest.mark.gpu


def _run_mask(gpu, orc, mask, sub, min_area=5, max_src=None):
    H, W = mask.shape
    ol, K, ost = orc.label(mask, sub, min_area, max_src=max_src)
    labels, n_src, st = gpu.detect_label(dev(sub), mask_in=dev(pack_mask(mask).view(np.int32)),
                                         min_area=min_area, max_src=max_src if max_src is not None else max(K, 1))
    torch.cuda.synchronize()
    gl = host(labels)
    assert int(host(n_src)[0]) == K
    assert np.array_equal(gl, ol), f"label map differs at {np.argwhere(gl != ol)[:5]}"
    n = min(K, max_src if max_src is not None else K)
    g = {k: host(v)[:n] for k, v in st.items()}
    for k in ("area", "first", "xmin", "xmax", "ymin", "ymax"):
        assert np.array_equal(g[k], ost[k][:n]), k
    assert np.array_equal(g["peak"], ost["peak"][:n].astype(np.float32))
    assert rel_close(g["flux"], ost["sum"][:n], 1e-5, 1e-6).all()
    # barycentres: FP32 products f * x (tile-relative x < 128), FP64 sums
    for k, o in (("xbar", "xbar"), ("ybar", "ybar")):
        tol = 2 * float_ulp(ost[o][:n]) + 2e-5
        assert np.all(np.abs(g[k] - ost[o][:n]) <= tol), k
    return K


@pytest.mark.parametrize("shape,p,seed", [((221, 300), 0.3, 1), ((64, 128), 0.5, 2), ((97, 513), 0.15, 3),
                                          ((33, 129), 0.6, 4), ((1, 700), 0.5, 5), ((700, 1), 0.5, 6),
                                          ((256, 256), 0.05, 7)])
def test_random_masks(gpu, orc, shape, p, seed):
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=shape) < p).astype(np.uint8)
    sub = rng.uniform(0.5, 100.0, shape).astype(np.float32)
    for min_area in (1, 5):
        _run_mask(gpu, orc, mask, sub, min_area)


def test_degenerate_masks(gpu, orc):
    H, W = 100, 300
    sub = np.random.default_rng(9).uniform(1, 2, (H, W)).astype(np.float32)
    assert _run_mask(gpu, orc, np.zeros((H, W), np.uint8), sub) == 0
    assert _run_mask(gpu, orc, np.ones((H, W), np.uint8), sub) == 1
    cb = (np.add.outer(np.arange(H), np.arange(W)) % 2).astype(np.uint8)   # 8-connected checkerboard
    assert _run_mask(gpu, orc, cb, sub, 1) == 1
    iso = np.zeros((H, W), np.uint8)
    iso[::2, ::2] = 1                                                      # isolated pixels
    assert _run_mask(gpu, orc, iso, sub, 1) == 50 * 150
    assert _run_mask(gpu, orc, iso, sub, 2) == 0
    one = np.zeros((H, W), np.uint8)
    one[99, 299] = 1
    assert _run_mask(gpu, orc, one, sub, 1) == 1


def test_spiral_across_tiles(gpu, orc):
    """one long snake that crosses many tile seams, plus diagonal-only links at
    tile corners (8-connectivity through a corner of four tiles)."""
    H, W = 160, 520
    m = np.zeros((H, W), np.uint8)
    for r in range(2, H - 2, 4):
        m[r, 2:W - 2] = 1
        c = W - 3 if (r // 4) % 2 == 0 else 2
        m[r:r + 4, c] = 1
    m[31, 127] = 1; m[32, 128] = 1; m[33, 129] = 1     # through the corner at (32, 128)
    m[31, 255] = 1; m[32, 254] = 1                     # anti-diagonal across a vertical seam
    sub = np.ones((H, W), np.float32)
    _run_mask(gpu, orc, m, sub, 1)
    _run_mask(gpu, orc, m, sub, 3)


def test_capacity(gpu, orc):
    mask = np.zeros((40, 200), np.uint8)
    mask[5:10, ::4] = 1        # 50 bars of area 5
    sub = np.ones(mask.shape, np.float32)
    assert _run_mask(gpu, orc, mask, sub, 5, max_src=7) == 50


def test_threshold_mode_matches_oracle_threshold(gpu, orc):
    """threshold computed on the GPU (FP32) vs the oracle (FP64): masks may differ
    only where sub is within rounding of k * rms(x, y); away from those pixels the
    label maps agree after renumbering by first pixel."""
    img, _ = synth.frame_gradient_1k(1001)
    ob, orr, _ = orc.bg_estimate(img, mesh=64)
    osub, _ = orc.bg_subtract(img, ob, 64)
    om = orc.threshold(osub, orr, 64, 1.5)
    rmsmap = orc.interp_map(orr, 64, 1024, 1024)
    labels, n_src, st = gpu.detect_label(dev(osub), dev(orr), mesh=64, k=1.5, min_area=5)
    gm = host(labels) > 0
    ol, K, _ = orc.label(om, osub, 5)
    near = np.abs(osub.astype(np.float64) - 1.5 * rmsmap) <= 1e-5 * np.abs(1.5 * rmsmap) + 1e-6
    diff = gm != (ol > 0)
    # a flipped pixel can only change membership of its own component
    assert diff.sum() <= 10 * max(near.sum(), 1)
    if near.sum() == 0:
        assert int(host(n_src)[0]) == K
        assert np.array_equal(host(labels), ol)


def test_survey_frame_full_size_labels(gpu, orc):
    """4096^2 survey field at the benchmark's sizes: with the oracle's mask the
    GPU label map over the whole frame is identical."""
    img, _ = synth.frame_survey_4k()
    ob, orr, _ = orc.bg_estimate(img, mesh=128)
    osub, _ = orc.bg_subtract(img, ob, 128)
    om = orc.threshold(osub, orr, 128, 1.5)
    K = _run_mask(gpu, orc, om, osub, 5)
    assert K > 10000


def test_mixed_dense_and_sparse_tiles(gpu, orc):
    """Tiles with more runs than the common pass holds (checkerboard and dense
    noise) next to ordinary tiles: the dense ones are redone by the
    full-capacity pass and the seams between the two kinds still merge."""
    H, W = 200, 700
    rng = np.random.default_rng(21)
    mask = (rng.uniform(size=(H, W)) < 0.08).astype(np.uint8)
    mask[:, :260] = (np.add.outer(np.arange(H), np.arange(260)) % 2).astype(np.uint8)
    mask[40:140, 400:530] = (rng.uniform(size=(100, 130)) < 0.55).astype(np.uint8)
    sub = rng.uniform(0.5, 50.0, (H, W)).astype(np.float32)
    for min_area in (1, 5):
        _run_mask(gpu, orc, mask, sub, min_area)


"""Whole-path sanity of the oracle against the generator's injected truth (the
paper's own accuracy levels, Sec. 3.3: ~98% of positions within 0.04 px and ~95%
of magnitudes within 0.04 of SExtractor, used here as loose levels against truth
for bright isolated stars) and calibration closed forms."""
import math

import numpy as np
import pytest

import synth
from metrics import match, recall_precision_f1


def test_calibrate_hand_values(orc):
    raw = np.array([[600, 500, 0, 65535]], np.uint16)
    flat = np.array([[0.5, 1.0, 2.0, 1.0]], np.float32)
    out = orc.calibrate(raw, flat, bias=500.0)
    assert out.tolist() == [[200.0, 0.0, -250.0, 65035.0]]
    bm = np.array([[100, 100, 100, 100]], np.float32)
    assert orc.calibrate(raw, flat, bias_map=bm).tolist() == [[1000.0, 400.0, -50.0, 65435.0]]


def test_metrics_reading():
    m = np.array([0, 1, -1, 2, -1])
    r, p, f1 = recall_precision_f1(m, 4)
    assert (r, p) == (0.75, 0.6) and f1 == pytest.approx(2 * 0.75 * 0.6 / 1.35)


def test_catalog_vs_truth_1k(orc):
    img, tr = synth.frame_gradient_1k()
    out = orc.catalog(img)
    assert 500 <= out["K"] < 2000
    # bright isolated stars (no other star within 12 px, 15 px from the edges)
    from scipy.spatial import cKDTree
    t = cKDTree(np.stack([tr.x, tr.y], 1))
    nn = np.array([len(t.query_ball_point([a, b], 12.0)) for a, b in zip(tr.x, tr.y)])
    inner = (tr.x > 15) & (tr.x < 1009) & (tr.y > 15) & (tr.y < 1009)
    sel = (tr.flux > 3e4) & (nn == 1) & inner   # SNR > 150: position noise ~0.01 px
    m, d = match(out["x"], out["y"], tr.x, tr.y)
    det = np.zeros(len(tr.x), bool)
    det[m[m >= 0]] = True
    assert det[sel].mean() > 0.99
    r, p, f1 = recall_precision_f1(m, len(tr.x))
    assert r > 0.8
    k = np.flatnonzero(m >= 0)
    k = k[sel[m[k]]]
    dpos = np.hypot(out["x"][k] - tr.x[m[k]], out["y"][k] - tr.y[m[k]])
    assert np.mean(dpos < 0.04) > 0.98
    s = 3.0 / (2 * math.sqrt(2 * math.log(2)))
    expect = tr.flux[m[k]] * (1 - math.exp(-25 / (2 * s * s)))
    dmag = -2.5 * np.log10(out["flux"][k] / expect)
    assert np.mean(np.abs(dmag) < 0.04) > 0.95


def test_spline_reading_of_the_catalog(orc):
    """the catalog with the natural-spline map: a constant sky is subtracted
    exactly (the spline of equal nodes is that value everywhere, the linear
    extension included) and nothing is detected; on a sky with stars the
    subtracted frame equals the frame less the oracle's spline map"""
    import synth
    f = np.full((200, 300), 500.0, np.float32)
    c = orc.catalog(f, mesh=32, interp="spline")
    assert c["K"] == 0 and np.all(c["sub"] == 0.0)
    img, _ = synth.tiny_frame(300, 200, 5, n_stars=8, sky=400.0)
    c = orc.catalog(img, mesh=32, interp="spline")
    B = orc.spline_map(c["bkg"], 32, 300, 200)
    assert np.array_equal(c["sub"], (img.astype(np.float64) - B).astype(np.float32))
    assert c["K"] >= 4

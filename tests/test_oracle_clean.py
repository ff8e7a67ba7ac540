"""Pins of the oracle's cleaning of deblended objects (Sec. 2.2.5; the reading
follows SExtractor's cleaning: each object's peak, less the Moffat models of the
brighter objects there, must reach the detection threshold, else it merges into
the largest contributor).  Pins: single-pixel objects, whose moments are the
1/12 of a uniform pixel, give closed-form model values -- 1 + 12 d^2 / a^2 to
the power -beta with a^2 = 2 ln 2 / (2^(1/beta) - 1), and the Gaussian exp(-6 d^2)
in the large-beta limit -- so the keep/merge decision flips exactly where they
say; isolated stars are all kept; a faint bump on a bright star's wing merges
and a bright one stays; the merge target is the largest contributor; the result
does not depend on the numbering of the objects."""
import math

import numpy as np
import pytest


def _two_pixels(v_faint, d=1):
    sub = np.zeros((21, 21), np.float32)
    lab = np.zeros((21, 21), np.int32)
    sub[10, 10], lab[10, 10] = 1e4, 1
    sub[10, 10 + d], lab[10, 10 + d] = v_faint, 2
    return sub, lab


@pytest.mark.parametrize("beta", [1.0, 2.5, 1e6])
def test_single_pixel_closed_form(orc, beta):
    thr = 10.0
    if beta > 1e5:
        model = 1e4 * math.exp(-6.0)            # the Gaussian limit, r^2 = 12 d^2, d = 1
    else:
        a2 = 2.0 * math.log(2.0) / (2.0 ** (1.0 / beta) - 1.0)
        model = 1e4 * (1.0 + 12.0 / a2) ** -beta
    edge = model + thr
    for v, merged in ((edge * (1 - 2e-5), True), (edge * (1 + 2e-5), False)):
        sub, lab = _two_pixels(v)
        out, k = orc.clean(sub, lab, 2, thr, beta=beta)
        assert k == (1 if merged else 2)
        assert out[10, 11] == (1 if merged else 2) and out[10, 10] == 1


def _gauss(H, W, stars):
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    img = np.zeros((H, W))
    for x, y, peak, s in stars:
        img += peak * np.exp(-((j - x) ** 2 + (i - y) ** 2) / (2 * s * s))
    return img


def test_isolated_stars_are_kept(orc):
    stars = [(15, 15, 500, 1.5), (60, 15, 800, 1.5), (15, 60, 300, 1.5), (60, 60, 1000, 1.5)]
    sub = _gauss(80, 80, stars).astype(np.float32)
    lab, K, _ = orc.label((sub > 20).astype(np.uint8), sub, min_area=1)
    out, k = orc.clean(sub, lab, K, 20.0)
    assert K == 4 and k == 4 and np.array_equal(out, lab)


@pytest.mark.parametrize("bump,merged", [(40.0, True), (200.0, False)])
def test_wing_bump(orc, bump, merged):
    """a bright star (peak 1000) and a 3 x 3 bump 9 px away: the broad beta = 1
    model of the star there is ~37, so a bump of 40 does not stand out by the
    threshold 20 and merges; a bump of 200 stays"""
    H = W = 60
    sub = _gauss(H, W, [(25, 30, 1000.0, 1.5)])
    lab = np.zeros((H, W), np.int32)
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    lab[(j - 25) ** 2 + (i - 30) ** 2 <= 36] = 1
    sub[29:32, 33:36] += bump * np.array([[0.5, 0.7, 0.5], [0.7, 1.0, 0.7], [0.5, 0.7, 0.5]])
    lab[29:32, 33:36] = 2
    out, k = orc.clean(sub.astype(np.float32), lab, 2, 20.0)
    assert k == (1 if merged else 2)
    assert np.array_equal(out > 0, lab > 0)
    assert np.all(out[lab == 2] == (1 if merged else 2))


def test_merge_target_is_the_largest_contributor(orc):
    """two bright single pixels at distances 2 and 3 from a faint one: the
    nearer one contributes more and takes it"""
    sub = np.zeros((15, 30), np.float32)
    lab = np.zeros((15, 30), np.int32)
    sub[7, 5], lab[7, 5] = 5e3, 1        # distance 3 from the faint pixel
    sub[7, 10], lab[7, 10] = 5e3, 2      # distance 2
    sub[7, 8], lab[7, 8] = 30.0, 3
    out, k = orc.clean(sub, lab, 3, 10.0)
    assert k == 2 and out[7, 8] == out[7, 10] == 2 and out[7, 5] == 1


def test_numbering_invariance(orc):
    rng = np.random.default_rng(6)
    stars = [(rng.uniform(5, 95), rng.uniform(5, 75), rng.uniform(30, 3000), rng.uniform(1.0, 2.0)) for _ in range(40)]
    sub = (_gauss(80, 100, stars) + rng.normal(0, 3.0, (80, 100))).astype(np.float32)
    lab, K, _ = orc.label((sub > 12).astype(np.uint8), sub, min_area=1)
    out, k = orc.clean(sub, lab, K, 12.0)
    perm = rng.permutation(K) + 1
    lab2 = np.where(lab > 0, perm[np.maximum(lab, 1) - 1], 0).astype(np.int32)
    out2, k2 = orc.clean(sub, lab2, K, 12.0)
    assert k2 == k and k < K
    # the same partition of the pixels
    pairs = np.unique(np.stack([out[lab > 0], out2[lab > 0]], 1), axis=0)
    assert len(pairs) == k and len(np.unique(pairs[:, 0])) == k and len(np.unique(pairs[:, 1])) == k


def test_object_statistics_brute_force(orc):
    """peak, barycentre and moments per object against a direct numpy evaluation"""
    rng = np.random.default_rng(9)
    sub = rng.normal(0, 5, (40, 50)).astype(np.float32)
    lab = np.zeros((40, 50), np.int32)
    lab[5:12, 5:15] = 1
    lab[20:30, 30:33] = 2
    lab[35, 40] = 3                       # one pixel
    sub[35, 40] = -2.0                    # with no positive value
    sub[5:12, 5:15] += 40.0
    st = orc.clean_stats(sub, lab, 3)
    for l in (1, 2, 3):
        i, j = np.nonzero(lab == l)
        f = sub[i, j].astype(np.float64)
        k = np.argmax(f)                   # first maximum in raster order
        assert st["peak"][l] == f[k] and st["peak_index"][l] == i[k] * 50 + j[k]
        w = np.maximum(f, 0.0)
        if w.sum() > 0:
            cx, cy = (w * j).sum() / w.sum(), (w * i).sum() / w.sum()
            x2, y2 = (w * (j - cx) ** 2).sum() / w.sum(), (w * (i - cy) ** 2).sum() / w.sum()
            xy = (w * (j - cx) * (i - cy)).sum() / w.sum()
            if x2 * y2 - xy * xy < 1 / 144:
                x2, y2 = x2 + 1 / 12, y2 + 1 / 12
        else:
            cx, cy, x2, y2, xy = j.mean(), i.mean(), 1 / 12, 1 / 12, 0.0
        got = [st[k2][l] for k2 in ("cx", "cy", "x2", "y2", "xy")]
        assert np.allclose(got, [cx, cy, x2, y2, xy], rtol=1e-12, atol=1e-12)


def test_empty_label_takes_no_number(orc):
    """a label with no pixel is no object: the objects on either side of it are
    numbered 1 and 2, and the count leaves it out"""
    sub = np.zeros((10, 30), np.float32)
    lab = np.zeros((10, 30), np.int32)
    sub[5, 3], lab[5, 3] = 100.0, 1
    sub[5, 25], lab[5, 25] = 100.0, 3     # label 2 has no pixel
    out, k = orc.clean(sub, lab, 3, 10.0)
    assert k == 2 and out[5, 3] == 1 and out[5, 25] == 2

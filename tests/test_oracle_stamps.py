"""Pins of the oracle's stamp cut (the input of the PSF fit; paper-silent reading
of Sec. 2.2.5's photometry): interior stamps equal numpy slices of the frame,
the centre pixel is the nearest one with ties rounded up, and pixels beyond
the frame are zero with zero weight and an EDGE flag."""
import numpy as np

EDGE = 1


def _frame(H, W, seed=0):
    return np.random.default_rng(seed).normal(size=(H, W)).astype(np.float32)


def test_interior_stamps_are_frame_slices(orc):
    img = _frame(60, 70)
    rng = np.random.default_rng(1)
    x = rng.uniform(8, 61, 50).astype(np.float32)
    y = rng.uniform(8, 51, 50).astype(np.float32)
    out = orc.stamp_cut(img, x, y, S=15)
    for s in range(50):
        cx, cy = int(np.floor(float(x[s]) + 0.5)), int(np.floor(float(y[s]) + 0.5))
        assert np.array_equal(out["stamps"][s], img[cy - 7:cy + 8, cx - 7:cx + 8])
        assert np.all(out["weights"][s] == 1.0)
        assert tuple(out["origin"][s]) == (cx - 7, cy - 7)
        assert out["flags"][s] == 0


def test_ties_round_up_and_negative_positions(orc):
    img = _frame(40, 40)
    x = np.array([10.5, 10.499999, 11.5, -0.5, -1.5, 9.0], np.float32)
    y = np.array([20.0, 20.0, 20.5, 20.0, 20.0, -0.5], np.float32)
    out = orc.stamp_cut(img, x, y, S=5)
    assert [tuple(o) for o in out["origin"]] == [(9, 18), (8, 18), (10, 19), (-2, 18), (-3, 18), (7, -2)]


def test_edge_fill_and_flags(orc):
    img = _frame(30, 25)
    x = np.array([0.0, 24.0, 12.0, 12.0, np.nan], np.float32)
    y = np.array([0.0, 29.0, 15.0, 40.0, 3.0], np.float32)
    out = orc.stamp_cut(img, x, y, S=7)
    assert list(out["flags"]) == [EDGE, EDGE, 0, EDGE, EDGE]
    # corner stamp: the lower-right 4 x 4 block is the frame's corner, the rest zero
    st, w = out["stamps"][0], out["weights"][0]
    assert np.array_equal(st[3:, 3:], img[:4, :4]) and np.all(w[3:, 3:] == 1)
    assert np.all(st[:3, :] == 0) and np.all(st[:, :3] == 0) and np.all(w[:3, :] == 0) and np.all(w[:, :3] == 0)
    # entirely outside / NaN: zeros, weight 0
    assert np.all(out["stamps"][3] == 0) and np.all(out["weights"][3] == 0)
    assert np.all(out["stamps"][4] == 0) and tuple(out["origin"][4]) == (0, 0)

"""Pins of the oracle's natural-spline background map (Sec. 2.2.2's spline
interpolation of the mesh, the natural cubic spline reading): scipy's natural
CubicSpline applied in the other axis order (the tensor-product spline does not
depend on it) inside the node hull; exact reproduction of linear and bilinear
node fields everywhere, the linear extension beyond the end nodes included;
the node values at node centres; the degenerate grids of one and two nodes."""
import numpy as np
from scipy.interpolate import CubicSpline


def _node_coords(n_pix, mesh):
    return (np.arange(n_pix) + 0.5) / mesh - 0.5


def test_matches_scipy_natural_spline_inside_hull(orc):
    rng = np.random.default_rng(1)
    ny, nx, mw, mh = 7, 9, 32, 24
    mesh = rng.normal(100.0, 5.0, (ny, nx)).astype(np.float32)
    W, H = nx * mw, ny * mh
    got = orc.spline_map(mesh, mw, W, H, mesh_h=mh)
    u, v = _node_coords(W, mw), _node_coords(H, mh)
    # y first (node columns), then x
    cols = CubicSpline(np.arange(ny), mesh.astype(np.float64), axis=0, bc_type="natural")(v)   # (H, nx)
    ref = CubicSpline(np.arange(nx), cols, axis=1, bc_type="natural")(u)                      # (H, W)
    inside = (v >= 0) & (v <= ny - 1)
    inside_x = (u >= 0) & (u <= nx - 1)
    sel = np.ix_(inside, inside_x)
    assert np.max(np.abs(got[sel] - ref[sel])) < 1e-10


def test_linear_and_bilinear_fields_are_exact(orc):
    ny, nx, m = 5, 6, 16
    q, p = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    mesh = (3.0 + 0.5 * q - 0.25 * p + 0.125 * p * q).astype(np.float32)   # exact in float32
    W, H = nx * m + 5, ny * m + 3                                           # pixels past the last node too
    got = orc.spline_map(mesh, m, W, H)
    u, v = _node_coords(W, m), _node_coords(H, m)
    uu, vv = np.meshgrid(u, v)
    assert np.max(np.abs(got - (3.0 + 0.5 * uu - 0.25 * vv + 0.125 * uu * vv))) < 1e-12


def test_node_values_at_node_centres(orc):
    rng = np.random.default_rng(2)
    mesh = rng.normal(0, 1, (4, 6)).astype(np.float32)
    m = 5                                   # node q sits at pixel 5 q + 2
    got = orc.spline_map(mesh, m, 6 * m, 4 * m)
    assert np.max(np.abs(got[2::m, 2::m] - mesh)) < 1e-12


def test_small_grids(orc):
    one = np.array([[7.0]], np.float32)
    assert np.all(orc.spline_map(one, 8, 10, 6) == 7.0)
    two = np.array([[1.0, 3.0]], np.float32)          # one row of two nodes: a line in x, constant in y
    got = orc.spline_map(two, 4, 8, 3)
    u = _node_coords(8, 4)
    assert np.max(np.abs(got - (1.0 + 2.0 * u)[None, :])) < 1e-12

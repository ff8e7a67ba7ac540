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


def test_node_second_derivatives_match_scipy(orc):
    """Mx, My and the cross term Mxy are the natural splines' second derivatives
    at the knots (scipy), and with the node values they give the map: the
    tensor form evaluated here from the 2 x 2 bracketing nodes equals the
    oracle's map inside the hull"""
    rng = np.random.default_rng(4)
    ny, nx, m = 6, 8, 16
    mesh = rng.normal(50.0, 3.0, (ny, nx)).astype(np.float32)
    Y = mesh.astype(np.float64)
    Mx, My, Mxy = orc.spline_nodes(mesh)
    kx, ky = np.arange(nx), np.arange(ny)
    assert np.allclose(Mx, CubicSpline(kx, Y, axis=1, bc_type="natural")(kx, 2), atol=1e-10)
    assert np.allclose(My, CubicSpline(ky, Y, axis=0, bc_type="natural")(ky, 2), atol=1e-10)
    assert np.allclose(Mxy, CubicSpline(ky, Mx, axis=0, bc_type="natural")(ky, 2), atol=1e-10)
    got = orc.spline_map(mesh, m, nx * m, ny * m)
    u, v = _node_coords(nx * m, m), _node_coords(ny * m, m)

    def w(t):      # weights of value, value, second derivative, second derivative on [k, k + 1]
        b = t - np.floor(t)
        a = 1 - b
        return a, b, (a ** 3 - a) / 6, (b ** 3 - b) / 6

    for ii in range(0, ny * m, 7):
        for jj in range(0, nx * m, 5):
            if not (0 <= u[jj] <= nx - 1 and 0 <= v[ii] <= ny - 1):
                continue
            q, p = min(int(u[jj]), nx - 2), min(int(v[ii]), ny - 2)
            ax, bx, cx, dx = w(u[jj] - q)
            ay, by, cy, dy = w(v[ii] - p)
            if u[jj] - q >= 1:
                ax, bx, cx, dx = 0.0, 1.0, 0.0, 0.0
            if v[ii] - p >= 1:
                ay, by, cy, dy = 0.0, 1.0, 0.0, 0.0

            def along_x(F, G, r):   # x-spline of row r from values F and x-derivatives G
                return ax * F[r, q] + bx * F[r, q + 1] + cx * G[r, q] + dx * G[r, q + 1]

            val = (ay * along_x(Y, Mx, p) + by * along_x(Y, Mx, p + 1)
                   + cy * along_x(My, Mxy, p) + dy * along_x(My, Mxy, p + 1))
            assert abs(val - got[ii, jj]) < 1e-10

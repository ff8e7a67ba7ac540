"""Pins of the oracle's PSF model, analytic Jacobian and Levenberg-Marquardt fit
(paper-silent readings) against finite differences, the model's closed-form
normalisation and peak, and scipy's MINPACK least-squares solver."""
import math

import numpy as np
import pytest
from scipy import optimize


def _rand_params(rng, S=15):
    c = (S - 1) / 2
    return np.array([c + rng.uniform(-0.6, 0.6), c + rng.uniform(-0.6, 0.6),
                     rng.uniform(500, 5e4), rng.uniform(50, 1000),
                     rng.uniform(1.0, 2.0), rng.uniform(1.0, 2.0), rng.uniform(-1.5, 1.5)])


@pytest.mark.parametrize("model", [0, 1], ids=["moffat", "gauss"])
def test_jacobian_vs_central_fd(orc, model):
    """analytic dm/dp vs central differences with h = 1e-3 (truncation O(h^2))."""
    rng = np.random.default_rng(20 + model)
    for _ in range(10):
        p = _rand_params(rng)
        m, J = orc.psf_model(p, 15, model)
        for k in range(7):
            h = 1e-3 * max(1.0, abs(p[k])) if k in (2, 3) else 1e-3
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            fd = (orc.psf_model(pp, 15, model, jac=False) - orc.psf_model(pm, 15, model, jac=False)) / (2 * h)
            scale = np.abs(J[:, k]).max() + 1e-30
            assert np.abs(fd.ravel() - J[:, k]).max() / scale < 2e-5, (k, model)


def test_model_closed_forms(orc):
    """Peak at a pixel-centred source: F (beta-1) / (pi sx sy) + sky (Moffat),
    F / (2 pi sx sy) + sky (Gaussian); a large stamp integrates to F (point
    sampling of a smooth profile; Moffat tail beyond the stamp < 1e-5 F)."""
    F, sky, sx, sy, b = 1e4, 7.0, 1.5, 1.2, 2.5
    p = np.array([7.0, 7.0, F, sky, sx, sy, 0.3])
    m = orc.psf_model(p, 15, 0, b, jac=False)
    assert m[7, 7] == pytest.approx(F * (b - 1) / (math.pi * sx * sy) + sky, rel=1e-14)
    m = orc.psf_model(p, 15, 1, jac=False)
    assert m[7, 7] == pytest.approx(F / (2 * math.pi * sx * sy) + sky, rel=1e-14)
    S = 401
    p = np.array([200.3, 199.8, F, 0.0, sx, sy, 0.7])
    assert orc.psf_model(p, S, 1, jac=False).sum() == pytest.approx(F, rel=1e-9)
    # Moffat: wide core (lattice sum = integral to ~exp(-2 pi alpha)) and beta = 4
    # (tail beyond the stamp (1 + R^2/alpha^2)^(1-beta) ~ 1e-11)
    p = np.array([200.3, 199.8, F, 0.0, 4.2, 4.0, 0.7])
    assert orc.psf_model(p, S, 0, 4.0, jac=False).sum() == pytest.approx(F, rel=1e-7)


def test_model_rotation_and_swap(orc):
    """(sx, sy, theta) and (sy, sx, theta + pi/2) describe the same image."""
    rng = np.random.default_rng(23)
    p = _rand_params(rng)
    q = p.copy()
    q[4], q[5], q[6] = p[5], p[4], p[6] + math.pi / 2
    for model in (0, 1):
        a = orc.psf_model(p, 15, model, jac=False)
        b = orc.psf_model(q, 15, model, jac=False)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-9)


def test_fit_noise_free_recovery(orc):
    rng = np.random.default_rng(24)
    for model in (0, 1):
        truth = np.array([_rand_params(rng) for _ in range(8)])
        truth[:, 4] = np.maximum(truth[:, 4], truth[:, 5] * 1.2)   # canonical: sx > sy
        stamps = np.array([orc.psf_model(t, 15, model, jac=False) for t in truth]).astype(np.float32)
        out = orc.psf_fit(stamps, model=model, max_iter=200)
        got = out["params"]
        assert np.all(out["flags"] == 0)
        assert np.allclose(got[:, :6], truth[:, :6], rtol=1e-4, atol=1e-4)
        dth = (got[:, 6] - truth[:, 6] + math.pi / 2) % math.pi - math.pi / 2
        assert np.abs(dth).max() < 1e-3


def test_fit_matches_minpack(orc):
    """Noisy stamps of well-measured stars (flux > 5e3 ADU, where the optimum is
    unique): the oracle's optimum agrees with scipy's MINPACK
    Levenberg-Marquardt started from the same point."""
    import synth
    stamps, truth = synth.moffat_stamps(60, seed=4321)
    keep = truth[:, 2] > 5e3
    stamps = stamps[keep][:10]
    assert len(stamps) >= 5
    out = orc.psf_fit(stamps, max_iter=200)
    assert np.all(out["flags"] == 0)
    for s in range(len(stamps)):
        p0 = orc.psf_init(stamps[s])

        def res(p):
            return (stamps[s].astype(np.float64) - orc.psf_model(p, 15, 0, jac=False)).ravel()

        def jac(p):
            return -orc.psf_model(p, 15, 0)[1]
        r = optimize.least_squares(res, p0, jac=jac, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                                   max_nfev=20000)
        c2 = float(np.sum(r.fun ** 2))
        assert out["chi2"][s] == pytest.approx(c2, rel=1e-6)
        q = r.x.copy()
        if q[4] < q[5]:
            q[4], q[5], q[6] = q[5], q[4], q[6] + math.pi / 2
        q[6] = q[6] - math.pi * math.floor((q[6] + math.pi / 2) / math.pi)
        assert np.allclose(out["params"][s, :6], q[:6], rtol=2e-4, atol=2e-4)


def test_fit_init_reading(orc):
    """Default start: stamp centre, border median as sky, sum above sky as flux,
    widths 1.6 / 1.4, angle 0."""
    st = np.full((15, 15), 3.0, np.float32)
    st[7, 7] = 103.0
    p = orc.psf_init(st)
    assert list(p) == [7.0, 7.0, 100.0, 3.0, 1.6, 1.4, 0.0]

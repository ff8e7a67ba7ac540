"""GPU parity of deblending (ipp_deblend) with the oracle from identical inputs
(subtracted frame, candidate label map and statistics).  The output is an
integer label map, so the bar is bit-exact: every decision is a comparison of
FP64 quantities (levels, node fluxes, Gaussian likelihoods) whose rounding
differences between the two sides (summation order, pow/exp last bits) would
have to land within ~1e-16 of a threshold to change a label."""
import math

import numpy as np
import pytest
import torch
from scipy.special import erf

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _cdf(t):
    return 0.5 * (1.0 + erf(t / math.sqrt(2.0)))


def _stars(H, W, stars, noise=0.0, seed=0):
    img = np.zeros((H, W))
    j, i = np.arange(W), np.arange(H)
    for x, y, F, s in stars:
        ex = _cdf((j + 0.5 - x) / s) - _cdf((j - 0.5 - x) / s)
        ey = _cdf((i + 0.5 - y) / s) - _cdf((i - 0.5 - y) / s)
        img += F * ey[:, None] * ex[None, :]
    if noise:
        img += np.random.default_rng(seed).normal(0, noise, img.shape)
    return img.astype(np.float32)


def _gpu_inputs(labels, st, K):
    keys = ("xmin", "xmax", "ymin", "ymax", "area", "xbar")
    return {k: dev(np.ascontiguousarray(st[k][:K], np.int32 if k != "xbar" else np.float32)) for k in keys}


def _both(gpu, orc, img, labels, st, K, **kw):
    o_map, o_K = orc.deblend(img, labels, K, **kw)
    n_src = torch.tensor([K], dtype=torch.int32, device="cuda")
    g_map, g_K = gpu.deblend(dev(img), dev(labels), n_src, _gpu_inputs(labels, st, K), **kw)
    return o_map, o_K, host(g_map), int(host(g_K)[0])


@pytest.mark.parametrize("scene", ["pair", "triple", "contrast", "crowded"])
def test_deblend_scenes(gpu, orc, scene):
    if scene == "pair":
        img = _stars(41, 51, [(21.0, 20.0, 1e5, 1.5), (27.0, 20.5, 1e5, 1.5)])
        cut = 5.0
    elif scene == "triple":
        img = _stars(60, 80, [(20.0, 20.0, 1e5, 1.4), (26.0, 21.0, 8e4, 1.4), (23.0, 26.0, 6e4, 1.4),
                              (60.0, 40.0, 5e4, 1.4)])
        cut = 5.0
    elif scene == "contrast":
        img = _stars(41, 61, [(20.0, 20.0, 1e5, 1.5), (30.0, 20.0, 1e4, 1.5)])
        cut = 0.5
    else:
        rng = np.random.default_rng(7)
        st_ = [(rng.uniform(5, 123), rng.uniform(5, 91), 10 ** rng.uniform(3, 5), rng.uniform(1.2, 2.0))
               for _ in range(60)]
        img = _stars(96, 128, st_, noise=2.0, seed=8)
        cut = 8.0
    labels, K, st = orc.label((img > cut).astype(np.uint8), img, min_area=3)
    for mc in (0.005, 0.05):
        o_map, o_K, g_map, g_K = _both(gpu, orc, img, labels, st, K, mincont=mc)
        assert g_K == o_K
        assert np.array_equal(g_map, o_map)


@pytest.mark.parametrize("which", ["gradient_1k", "survey_4k"])
def test_deblend_frames(gpu, orc, which):
    """the GPU catalog of a frame (labels and statistics of ipp_extract),
    deblended on both sides; the survey frame is the benchmark's workload."""
    if which == "gradient_1k":
        img, _ = synth.frame_gradient_1k(1001)
        mesh = 64
    else:
        img, _ = synth.frame_survey_4k()
        mesh = 128
    out = gpu.extract(dev(img), mesh=mesh)
    K = int(host(out["n_src"])[0])
    sub, labels = host(out["sub"]), host(out["labels"])
    st = {k: host(out["stats"][k])[:K] for k in ("xmin", "xmax", "ymin", "ymax", "area", "xbar")}
    o_map, o_K = orc.deblend(sub, labels, K)
    g_map, g_K = gpu.deblend(out["sub"], out["labels"], out["n_src"], out["stats"], max_src=K)
    g_map, g_K = host(g_map), int(host(g_K)[0])
    assert g_K == o_K and g_K >= K
    assert np.array_equal(g_map, o_map)


def test_deblend_edge_cases(gpu, orc):
    img = _stars(30, 40, [(1.0, 1.0, 5e4, 1.3), (4.0, 1.5, 5e4, 1.3), (30.0, 20.0, 2e4, 1.3)])
    labels, K, st = orc.label((img > 5.0).astype(np.uint8), img, min_area=1)
    o_map, o_K, g_map, g_K = _both(gpu, orc, img, labels, st, K)
    assert g_K == o_K and np.array_equal(g_map, o_map)
    # capacity: only the first candidate is processed, the rest stays 0
    n_src = torch.tensor([K], dtype=torch.int32, device="cuda")
    g1, k1 = gpu.deblend(dev(img), dev(labels), n_src, _gpu_inputs(labels, st, K), max_src=1)
    g1 = host(g1)
    assert np.array_equal(g1 > 0, labels == 1)
    o1, ok1 = orc.deblend(img, np.where(labels == 1, 1, 0).astype(np.int32), 1)
    assert int(host(k1)[0]) == ok1 and np.array_equal(g1, o1)
    # empty catalog
    zero = torch.zeros(1, dtype=torch.int32, device="cuda")
    g0, k0 = gpu.deblend(dev(img), dev(labels), zero, _gpu_inputs(labels, st, K))
    assert int(host(k0)[0]) == 0 and not host(g0).any()

"""GPU parity of the stamp cut: a pure copy, so stamps, weights, origins and
flags must match the oracle exactly, including ties, edges and the device-side
source count."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def test_stamp_cut_exact(gpu, orc):
    img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0)
    rng = np.random.default_rng(5)
    n = 3000
    x = rng.uniform(-10, 527, n).astype(np.float32)
    y = rng.uniform(-10, 399, n).astype(np.float32)
    x[:40] = np.floor(x[:40]) + 0.5           # ties
    x[40], y[41] = np.nan, np.inf
    x[42] = 3e9
    o = orc.stamp_cut(img, x, y, S=15)
    g = gpu.stamp_cut(dev(img), dev(x), dev(y), S=15)
    for k in ("stamps", "weights", "origin", "flags"):
        assert np.array_equal(host(g[k]), o[k]), k


def test_stamp_cut_device_count_and_sizes(gpu, orc):
    img, _ = synth.frame_gradient_1k(1001)
    x = np.array([5.2, 500.7, 1020.0, 300.5], np.float32)
    y = np.array([7.9, 3.4, 1019.6, 600.5], np.float32)
    n_dev = torch.tensor([3], dtype=torch.int32, device="cuda")
    for S in (3, 15, 31):
        o = orc.stamp_cut(img, x[:3], y[:3], S=S)
        g = gpu.stamp_cut(dev(img), dev(x), dev(y), n_src=n_dev, S=S, max_src=4)
        assert np.array_equal(host(g["stamps"])[:3], o["stamps"])
        assert np.array_equal(host(g["flags"])[:3], o["flags"])

"""GPU parity of cleaning (ipp_clean; Sec. 2.2.5, the reading after
SExtractor's cleaning) with the oracle's orc_clean, from identical inputs.

Where the two sides can differ, and the bar that follows: the peaks and their
pixels are maxima of the same FP32 values on both sides (exact); the
barycentres and moments come from exact integer sums on the GPU and FP64 sums in
the oracle (equal to ~1e-7 relative); the models and the test are FP32 on the
GPU, so each model value is within ~1e-6 relative of the oracle's.  A decision
can then differ only for an object whose margin pk - sum - thr lies within
1e-5 (|pk| + sum + |thr|) of zero, and a merge target only where the two
largest models are within 1e-5 of each other.  Such objects are *ambiguous*.
Every object whose merge chain (in the oracle) passes through no ambiguous
object ends at the same kept object on both sides; with no ambiguous object the
label maps are identical."""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _decisions(orc, sub, labels, n, thr_map, beta):
    """Per label (FP64, from the oracle's statistics): merge target (itself when
    kept), ambiguity flag, peak and peak pixel."""
    st = orc.clean_stats(sub, labels, n)
    pk, pidx = st["peak"], st["peak_index"]
    valid = pidx >= 0
    valid[0] = False
    W = sub.shape[1]
    a2 = 2.0 * math.log(2.0) / (2.0 ** (1.0 / beta) - 1.0)
    det = st["x2"] * st["y2"] - st["xy"] ** 2
    into = np.arange(n + 1)
    amb = np.zeros(n + 1, bool)
    idx = np.flatnonzero(valid)
    jj = np.arange(n + 1)
    thr_flat = thr_map.ravel()
    for c0 in range(0, idx.size, 512):
        ii = idx[c0:c0 + 512]
        px, py = (pidx[ii] % W).astype(np.float64), (pidx[ii] // W).astype(np.float64)
        dx = px[:, None] - st["cx"][None, :]
        dy = py[:, None] - st["cy"][None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            r2 = (st["y2"] * dx * dx - 2.0 * st["xy"] * dx * dy + st["x2"] * dy * dy) / det
            m = pk[None, :] * (1.0 + r2 / a2) ** -beta
        brighter = (pk[None, :] > pk[ii, None]) | ((pk[None, :] == pk[ii, None]) & (jj[None, :] < ii[:, None]))
        brighter &= valid[None, :] & (jj[None, :] != ii[:, None])
        m = np.where(brighter, m, -1.0)
        s = np.where(brighter, m, 0.0).sum(1)
        best = m.argmax(1)
        top2 = -np.sort(-m, axis=1)[:, :2] if m.shape[1] > 1 else np.c_[m, m]
        has = brighter.any(1)
        thr = thr_flat[pidx[ii]].astype(np.float64)
        margin = pk[ii] - s - thr
        merged = has & (margin < 0)
        into[ii[merged]] = best[merged]
        amb_dec = np.abs(margin) <= TOL * (np.abs(pk[ii]) + s + np.abs(thr))
        amb_tgt = (top2[:, 1] >= top2[:, 0] * (1.0 - TOL)) & (top2[:, 1] > 0)
        amb[ii] = has & (amb_dec | (amb_tgt & (merged | amb_dec)))
    return into, amb, pk, pidx, valid


def _roots_from_map(m, pk, pidx, valid):
    """label -> kept object (the brightest of its group: merges go to strictly
    brighter objects, so a group's kept object is its brightest) and the check that
    the kept objects are numbered 1.. in label order"""
    n = pk.size - 1
    new = np.zeros(n + 1, np.int64)
    new[valid] = m.ravel()[pidx[valid]]
    root = np.zeros(n + 1, np.int64)
    groups = {}
    for l in np.flatnonzero(valid):
        groups.setdefault(int(new[l]), []).append(int(l))
    kept = []
    for g, members in groups.items():
        r = max(members, key=lambda l: (pk[l], -l))
        root[members] = r
        kept.append((r, g))
    kept.sort()
    assert [g for _, g in kept] == list(range(1, len(kept) + 1)), "kept objects not numbered in label order"
    return root


def _chain_clean(into, amb, valid):
    n = into.size - 1
    ok = np.zeros(n + 1, bool)
    for i in np.flatnonzero(valid):
        r, good = i, not amb[i]
        while into[r] != r and good:
            r = into[r]
            good = not amb[r]
        ok[i] = good
    return ok


def _compare(orc, sub, labels, n, thr_map, beta, g_map, g_k, max_obj=None):
    nn = n if max_obj is None else min(n, max_obj)
    o_map, o_k = orc.clean(sub, labels, nn, thr_map, beta=beta)
    into, amb, pk, pidx, valid = _decisions(orc, sub, labels, nn, thr_map, beta)
    o_root = _roots_from_map(o_map, pk, pidx, valid)
    g_root = _roots_from_map(g_map, pk, pidx, valid)
    ok = _chain_clean(into, amb, valid)
    # the test-side decisions reproduce the oracle's map (FP64 on both)
    chain = np.arange(nn + 1)
    for i in np.flatnonzero(valid & ok):
        r = i
        while into[r] != r:
            r = into[r]
        chain[i] = r
    assert np.array_equal(chain[valid & ok], o_root[valid & ok])
    bad = np.flatnonzero(valid & ok & (g_root != o_root))
    assert bad.size == 0, f"{bad.size} objects end at another kept object, e.g. label {bad[:5]}"
    n_amb = int(amb.sum())
    assert abs(g_k - o_k) <= n_amb
    if n_amb == 0:
        assert g_k == o_k and np.array_equal(g_map, o_map)
    return dict(n=nn, oK=o_k, gK=g_k, ambiguous=n_amb, merged=int(nn - o_k))


def _gpu_clean(gpu, sub, labels, n, beta, thr_map=None, thresh_abs=0.0, max_obj=None, **kw):
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    m, k = gpu.clean(sub, labels, n_dev, n if max_obj is None else max_obj, thr_map=thr_map,
                     thresh_abs=thresh_abs, beta=beta, **kw)
    return host(m), int(host(k)[0])


def _stars(H, W, stars, noise=0.0, seed=0):
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    img = np.zeros((H, W))
    for x, y, peak, s in stars:
        img += peak * np.exp(-((j - x) ** 2 + (i - y) ** 2) / (2 * s * s))
    if noise:
        img += np.random.default_rng(seed).normal(0, noise, img.shape)
    return img.astype(np.float32)


def _scene(name):
    rng = np.random.default_rng(11)
    if name == "bumps":
        # bright stars with faint and bright satellites on their wings
        st = []
        for k in range(12):
            x, y = 20 + 40 * (k % 4), 20 + 40 * (k // 4)
            st.append((x, y, 1000.0 * (1 + k), 1.6))
            st.append((x + 7 + rng.uniform(-1, 1), y + rng.uniform(-2, 2), rng.uniform(20, 400), 1.0))
        return _stars(120, 170, st, noise=1.0, seed=3), 15.0
    if name == "crowded":
        st = [(rng.uniform(5, 250), rng.uniform(5, 250), 10 ** rng.uniform(2, 4.5), rng.uniform(1.0, 2.2))
              for _ in range(260)]
        return _stars(256, 256, st, noise=2.0, seed=5), 10.0
    st = [(rng.uniform(5, 380), rng.uniform(5, 200), 10 ** rng.uniform(1.7, 3.5), rng.uniform(0.8, 1.5))
          for _ in range(150)]
    return _stars(210, 389, st, noise=1.0, seed=6), 6.0   # ragged width


@pytest.mark.parametrize("beta", [1.0, 2.5])
@pytest.mark.parametrize("scene", ["bumps", "crowded", "ragged"])
def test_clean_scenes(gpu, orc, scene, beta):
    """deblended scenes (oracle deblending of the thresholded frame), constant threshold"""
    img, cut = _scene(scene)
    labels, K, _ = orc.label((img > cut).astype(np.uint8), img, min_area=1)
    dl, n = orc.deblend(img, labels, K)
    g_map, g_k = _gpu_clean(gpu, dev(img), dev(dl), n, beta, thresh_abs=cut)
    thr = np.full(img.shape, cut, np.float32)
    r = _compare(orc, img, dl, n, thr, beta, g_map, g_k)
    assert r["n"] > 10
    if beta == 1.0:
        assert r["merged"] > 0


def test_clean_threshold_map(gpu, orc):
    """a threshold map read at each object's peak pixel"""
    img, cut = _scene("crowded")
    labels, K, _ = orc.label((img > cut).astype(np.uint8), img, min_area=1)
    dl, n = orc.deblend(img, labels, K)
    yy, xx = np.mgrid[0:img.shape[0], 0:img.shape[1]]
    thr = (cut * (0.5 + xx / img.shape[1] + 0.3 * np.sin(yy / 17.0))).astype(np.float32)
    g_map, g_k = _gpu_clean(gpu, dev(img), dev(dl), n, 1.0, thr_map=dev(thr))
    _compare(orc, img, dl, n, thr, 1.0, g_map, g_k)


@pytest.mark.parametrize("which", ["gradient_1k", "survey_4k"])
def test_clean_frames(gpu, orc, which):
    """the GPU catalog of a frame, deblended, cleaned with the detection
    threshold (k rms interpolated from the mesh rms); the survey frame is the
    benchmark's workload"""
    if which == "gradient_1k":
        img, _ = synth.frame_gradient_1k(1001)
        mesh = 64
    else:
        img, _ = synth.frame_survey_4k()
        mesh = 128
    out = gpu.extract(dev(img), mesh=mesh)
    K = int(host(out["n_src"])[0])
    d_map, d_k = gpu.deblend(out["sub"], out["labels"], out["n_src"], out["stats"], max_src=K)
    n = int(host(d_k)[0])
    m, k = gpu.clean(out["sub"], d_map, d_k, n, mesh_rms=out["mesh_rms"], mesh=mesh, k=1.5)
    sub, dl = host(out["sub"]), host(d_map)
    H, W = sub.shape
    thr = np.maximum(1.5 * orc.interp_map(host(out["mesh_rms"]), mesh, W, H), 0.0).astype(np.float32)
    r = _compare(orc, sub, dl, n, thr, 1.0, host(m), int(host(k)[0]))
    assert r["n"] >= K


def test_clean_repeatable(gpu):
    """the sums are exact: two runs give the same map bit for bit"""
    img, _ = synth.frame_gradient_1k(1001)
    out = gpu.extract(dev(img), mesh=64)
    K = int(host(out["n_src"])[0])
    d_map, d_k = gpu.deblend(out["sub"], out["labels"], out["n_src"], out["stats"], max_src=K)
    n = int(host(d_k)[0])
    a = gpu.clean(out["sub"], d_map, d_k, n, mesh_rms=out["mesh_rms"], mesh=64)
    b = gpu.clean(out["sub"], d_map, d_k, n, mesh_rms=out["mesh_rms"], mesh=64)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_clean_edge_cases(gpu, orc):
    # single-pixel objects: the decision flips where the closed form says
    for beta in (1.0, 2.5):
        a2 = 2.0 * math.log(2.0) / (2.0 ** (1.0 / beta) - 1.0)
        edge = 1e4 * (1.0 + 12.0 / a2) ** -beta + 10.0
        for v, merged in ((edge * (1 - 2e-4), True), (edge * (1 + 2e-4), False)):
            sub = np.zeros((21, 21), np.float32)
            lab = np.zeros((21, 21), np.int32)
            sub[10, 10], lab[10, 10] = 1e4, 1
            sub[10, 11], lab[10, 11] = v, 2
            g, k = _gpu_clean(gpu, dev(sub), dev(lab), 2, beta, thresh_abs=10.0)
            assert k == (1 if merged else 2) and g[10, 11] == (1 if merged else 2) and g[10, 10] == 1
    # equal peaks: the smaller label is the brighter one; a negative-only object
    sub = np.zeros((30, 40), np.float32)
    lab = np.zeros((30, 40), np.int32)
    sub[10, 10:12], lab[10, 10:12] = 500.0, 1
    sub[10, 13:15], lab[10, 13:15] = 500.0, 2
    sub[20, 30:33], lab[20, 30:33] = -5.0, 3
    thr = np.full(sub.shape, 400.0, np.float32)
    g, k = _gpu_clean(gpu, dev(sub), dev(lab), 3, 1.0, thresh_abs=400.0)
    _compare(orc, sub, lab, 3, thr, 1.0, g, k)
    # capacity: labels above max_obj are background
    g, k = _gpu_clean(gpu, dev(sub), dev(lab), 3, 1.0, thresh_abs=400.0, max_obj=2)
    _compare(orc, sub, lab, 3, thr, 1.0, g, k, max_obj=2)
    assert not g[20].any()
    # no objects
    g, k = _gpu_clean(gpu, dev(sub), dev(lab), 0, 1.0, thresh_abs=400.0)
    assert k == 0 and not g.any()
    # an empty label between two objects
    lab2 = np.where(lab == 2, 3, np.where(lab == 3, 0, lab)).astype(np.int32)
    g, k = _gpu_clean(gpu, dev(sub), dev(lab2), 3, 1.0, thresh_abs=400.0)
    _compare(orc, sub, lab2, 3, thr, 1.0, g, k)


def test_clean_rejects_bad_args(gpu):
    sub = dev(np.zeros((8, 8), np.float32))
    lab = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(Exception):
        gpu.clean(sub, lab, n, 1, beta=0.0)
    with pytest.raises(Exception):
        gpu.clean(sub, lab, n, -1)

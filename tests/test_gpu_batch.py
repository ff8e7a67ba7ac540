"""The batched form of the catalog path (ipp_batch_*): frames of mixed sizes in
the table form (one launch per stage over a device table of all frames) and
spread over several streams, and the same batch replayed from a captured CUDA
graph, against per-frame ipp_extract calls on the same frames and against the
oracle frame by frame.  Every output must equal the per-frame call's bit for
bit: both run the same kernel bodies on the same inputs, and the labeling's
component sums are exact integer sums, independent of the order of the adds."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _frames():
    shapes = [(517, 389), (1024, 1024), (300, 221), (777, 640), (256, 256)]
    out = []
    for i, (W, H) in enumerate(shapes):
        img, _ = synth.tiny_frame(W, H, 300 + i, n_stars=30 + 10 * i, sky=400.0 + 50 * i)
        out.append(dev(img))
    return out


def _single(gpu, frames, **kw):
    res = []
    for f in frames:
        H, W = f.shape
        ex = gpu.Extractor(W, H, gpu.BgConfig(mesh=64), max_src=4096, **kw)
        o = ex(f)
        res.append({k: v.clone() for k, v in o.items()})
    torch.cuda.synchronize()
    return res


def _same(a, b):
    assert int(host(a["n_src"])[0]) == int(host(b["n_src"])[0])
    n = int(host(a["n_src"])[0])
    for k in ("labels", "mesh_bkg", "mesh_rms", "sub"):
        assert np.array_equal(host(a[k]), host(b[k])), k
    for k in ("x", "y", "flux", "sky", "area", "n_ann", "cen_flags", "phot_flags"):
        assert np.array_equal(host(a[k])[:n], host(b[k])[:n], equal_nan=True), k


@pytest.mark.parametrize("mode,lanes", [("streams", 1), ("streams", 3), ("table", 1)])
def test_batch_matches_single_frames(gpu, mode, lanes):
    frames = _frames()
    ref = _single(gpu, frames)
    b = gpu.Batch(frames, lanes=lanes, cfg=gpu.BgConfig(mesh=64), max_src=4096, mode=mode)
    outs = b.run()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        _same(o, r)
    b.close()


@pytest.mark.parametrize("mode", ["streams", "table"])
def test_batch_graph_replay_follows_inputs(gpu, mode):
    frames = _frames()
    b = gpu.Batch(frames, lanes=4, cfg=gpu.BgConfig(mesh=64), max_src=4096, mode=mode)
    b.run()  # one uncaptured run first: one-time kernel set-up happens outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    b.capture(s)
    for rep in range(2):
        for i, f in enumerate(frames):  # new contents, same buffers
            img, _ = synth.tiny_frame(f.shape[1], f.shape[0], 900 + 10 * rep + i, n_stars=25, sky=600.0)
            f.copy_(dev(img))
        torch.cuda.synchronize()
        ref = _single(gpu, frames)
        b.launch(s)
        s.synchronize()
        for o, r in zip(b.outs, ref):
            _same(o, r)
    b.close()


def test_batch_autotune_picks_a_lane_count(gpu):
    frames = _frames()[:3]
    b = gpu.Batch(frames, lanes=2, cfg=gpu.BgConfig(mesh=64), max_src=4096)
    best, ms = b.autotune()
    assert best in (1, 2, 4, 8) and all(m > 0 for m in ms)
    b.close()


@pytest.mark.parametrize("mode", ["streams", "table"])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle(gpu, orc, graph, mode):
    """every frame of a mixed batch (plain run, and the captured graph replayed)
    against the oracle's whole path on that frame: the matched-catalog
    comparison of the per-frame tests, frame by frame."""
    from catalog_match import assert_catalog
    from test_gpu_extract import host_catalog
    frames = _frames()
    b = gpu.Batch(frames, lanes=3, cfg=gpu.BgConfig(mesh=64), max_src=4096, mode=mode)
    b.run()
    torch.cuda.synchronize()
    if graph:
        s = torch.cuda.Stream()
        b.capture(s)
        for o in b.outs:  # the replay must rewrite every output
            o["labels"].fill_(-1)
            o["x"].fill_(float("nan"))
        b.launch(s)
        s.synchronize()
    for i, f in enumerate(frames):
        img = host(f)
        oc = orc.catalog(img, mesh=64)
        g, st = host_catalog(b.outs[i], b.stats[i])
        summ = assert_catalog(orc, img, oc, g, st, 64)
        assert summ["matched"] >= 0.97 * summ["oK"], (i, summ)
    b.close()


def test_table_rerun_and_mixed_sizes(gpu):
    """the table form run twice in a row (the second run reuses the uploaded
    table) on frames that span one to many labeling tiles, a calibrated raw
    frame among them"""
    shapes = [(31, 17), (2048, 1536), (129, 1000), (640, 480)]
    frames = []
    for i, (W, H) in enumerate(shapes):
        img, _ = synth.tiny_frame(W, H, 700 + i, n_stars=5 + 40 * i, sky=500.0)
        frames.append(dev(img))
    ref = _single(gpu, frames)
    b = gpu.Batch(frames, cfg=gpu.BgConfig(mesh=64), max_src=4096, mode="table")
    for _ in range(2):
        for o in b.outs:
            o["labels"].fill_(-1)
        b.run()
        torch.cuda.synchronize()
        for o, r in zip(b.outs, ref):
            _same(o, r)
    b.close()


def test_table_rejects_wide_centroid_window(gpu):
    frames = _frames()[:2]
    b = gpu.Batch(frames, cfg=gpu.BgConfig(mesh=64), max_src=4096, mode="table", fwhm_win=6.0)
    with pytest.raises(Exception):
        b.run()
    b.close()


def test_spline_reading_in_both_forms(gpu):
    """interp = spline: the stream form runs it (through ipp_extract, equal to the
    per-frame call); the table form answers NOT_SUPPORTED"""
    frames = _frames()[:3]
    cfg = gpu.BgConfig(mesh=64, interp="spline")
    ref = []
    for f in frames:
        ex = gpu.Extractor(f.shape[1], f.shape[0], cfg, max_src=4096)
        ref.append({k: v.clone() for k, v in ex(f).items()})
    b = gpu.Batch(frames, lanes=2, cfg=cfg, max_src=4096)
    b.run()
    torch.cuda.synchronize()
    for o, r in zip(b.outs, ref):
        _same(o, r)
    b.close()
    t = gpu.Batch(frames, cfg=cfg, max_src=4096, mode="table")
    with pytest.raises(Exception):
        t.run()
    t.close()


def test_table_raw_u16_with_bias_map(gpu):
    """raw uint16 frames with a bias map and a flat fused into every read, in the
    table form and per frame: every output equal bit for bit"""
    from test_gpu_extract import _raw_u16, _u16_tensor
    frames = []
    calib = None
    for i in range(3):
        raw, flat, bm = _raw_u16(6100 + i, W=640, H=480, n_stars=80, with_bias_map=True)
        frames.append(_u16_tensor(raw))
        if calib is None:   # one calibration for the batch (the frames share the flat and the bias map)
            calib = (dev((1.0 / flat.astype(np.float64)).astype(np.float32)), 500.0, dev(bm))
    ref = []
    for f in frames:
        ex = gpu.Extractor(640, 480, gpu.BgConfig(mesh=64), max_src=4096)
        ref.append({k: v.clone() for k, v in ex(f, calib).items()})
    b = gpu.Batch(frames, cfg=gpu.BgConfig(mesh=64), max_src=4096, mode="table", calib=calib)
    b.run()
    torch.cuda.synchronize()
    for o, r in zip(b.outs, ref):
        _same(o, r)
    b.close()

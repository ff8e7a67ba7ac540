"""Benchmark of the catalog path on one survey-sized frame per GPU.

Workload (per step, per GPU): one 4096 x 4096 float32 field -- sky 800..1200 ADU
with a quadratic variation, 20,000 stars (FWHM 2.5..4 px, power-law fluxes
1e2..1e6 ADU), 0.01% hot pixels, 200 cosmic rays -- through the whole catalog
path: mesh background (128 px meshes, 3x3 filter), interpolation + subtraction
fused with the 1.5 sigma threshold and the tile labeling, label merge and
numbering, windowed centroids and aperture photometry (r = 5, annulus 8-12).
Inputs stay resident in HBM; three frame copies rotate so that every step reads
a frame that is not in L2 (3 x 64 MiB > 129 MB).  A second leg fits 200,000
elliptical Moffat stamps of 15 x 15 px (batched LM) and reports stamps/s.

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle
on a bounded 1024 x 1024 crop of the same field instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MESH = 128
W = H = 4096
METRIC = "Mpix/s end-to-end per GB300 (catalog path, 4096^2 survey frame)"
WORKLOAD = ("survey_4k: 4096x4096 float32 field, 20,000 stars, hot pixels, cosmic rays; "
            "mesh 128, 3x3 filter, k=1.5, min_area 5, r=5, annulus 8-12")
# kernels ipp_extract launches per frame: mesh statistics, mesh filter,
# subtract+threshold, tile labeling, seam union, resolve, count, scan, emit,
# label map, centroid, aperture (plus one memset of the counters)
KERNELS_PER_FRAME = 12


def profiled_traffic(kernel_src, profile):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the source as it is now (the summary records the file's sha256); else None."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, profile)).read()
        digest = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()
    except OSError:
        return None
    if digest not in text:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    return int(m.group(1)) if m else None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def max_over_ranks(ms, ws, device):
    """Slowest replica's time: the whole job is done when the last rank is."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, ws, ms):
    """Aggregate throughput of all replicas (weak scaling: each rank processes
    units_per_step every step) over the slowest rank's time in ms."""
    return ws * steps * units_per_step / (ms / 1e3)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_all_cores():
    """The oracle's OpenMP build on every core this process may use (the same
    source and arithmetic; meshes, rows, sources and stamps spread over threads,
    CCL serial).  Returns the thread count, or 1 when OpenMP cannot be built."""
    import oracle
    n = host_cores()
    if n > 1:
        try:
            oracle.use_openmp(n)
        except Exception:
            return 1
    return n


def cpu_reference(steps, warmup, img=None, cores=None):
    """The FP64 oracle, as it stands, on the full 4096 x 4096 survey frame per
    step, on all host cores (cores = the threads it used)."""
    import oracle
    import synth
    if cores is None:
        cores = oracle_all_cores()
    if img is None:
        img, _ = synth.frame_survey_4k()
    for k in range(warmup):
        oracle.catalog(img, mesh=MESH)
    t0 = time.perf_counter()
    nsrc = 0
    for k in range(steps):
        nsrc += oracle.catalog(img, mesh=MESH)["K"]
    dt = time.perf_counter() - t0
    return dict(value=steps * W * H / 1e6 / dt, sec=dt, sources_per_s=nsrc / dt, steps=steps, cores=cores,
                sample=f"{steps} full 4096^2 survey frames, mesh {MESH}, OpenMP build on {cores} threads")


def cpu_single_core(img, n=4):
    """The plain (single-threaded) oracle on 1024^2 crops of the frame."""
    import numpy as np

    import oracle
    crops = [np.ascontiguousarray(img[r:r + 1024, c:c + 1024]) for r, c in
             [(0, 0), (1024, 2048), (2048, 1024), (3072, 3072)]]
    t0 = time.perf_counter()
    nsrc = 0
    for k in range(n):
        nsrc += oracle.catalog(crops[k % 4], mesh=MESH)["K"]
    dt = time.perf_counter() - t0
    return {"value": n * 1024 * 1024 / 1e6 / dt, "unit": "Mpix/s", "cores": 1, "sources_per_s": nsrc / dt,
            "sample": f"{n} crops of 1024x1024 px of the survey frame, plain build"}


def batch_leg(ipp, synth, dev, n_frames, reps=5, shapes=None, mesh=128, star_scale=1.0):
    """Frames of 2048^2, 4096^2 and 6144 x 6160 px (by index mod 3), 2,000-50,000
    stars and sky 200-3000 ADU each, drawn on the device: the per-frame path
    (one ipp_extract per frame on one stream) against the batch runner replayed
    from a captured CUDA graph, lanes chosen by its autotuner."""
    import numpy as np
    import torch
    shapes = shapes or synth.mixed_batch_shapes(n_frames)
    rng = np.random.default_rng(3000)
    frames = []
    for i, (W, H) in enumerate(shapes):
        n_st = max(1, int(rng.integers(2000, 50001) * star_scale))
        sky = float(rng.uniform(200.0, 3000.0))
        frames.append(synth.frame_field_device(W, H, n_st, 3000 + i, sky_level=sky, device=dev))
    cfg = ipp.BgConfig(mesh=mesh)
    exs = {}
    for f in frames:
        key = tuple(f.shape)
        if key not in exs:
            exs[key] = ipp.Extractor(f.shape[1], f.shape[0], cfg, device=dev, max_src=65536)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, st):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    per_ms = timed(lambda: [exs[tuple(f.shape)](f) for f in frames], stream)
    tuner = ipp.Batch(frames, lanes=1, cfg=cfg, max_src=65536)
    best, lane_ms = tuner.autotune()
    tuner.close()
    gs = torch.cuda.Stream(dev)
    # the stream form at its best lane count, plain and as a graph
    b = ipp.Batch(frames, lanes=best, cfg=cfg, max_src=65536)
    streams_ms = timed(lambda: b.run(gs), gs)
    b.capture(gs)
    streams_graph_ms = timed(lambda: b.launch(gs), gs)
    b.close()
    del b
    # the table form: one launch per stage over each lane group's frames, at
    # 1, 2, 4 and 8 lane groups (plain), then the best as a graph
    table_lane_ms = {}
    for tl in (1, 2, 4, 8):
        t = ipp.Batch(frames, lanes=tl, cfg=cfg, max_src=65536, mode="table")
        table_lane_ms[tl] = timed(lambda: t.run(gs), gs)
        t.close()
        del t
    tbest = min(table_lane_ms, key=table_lane_ms.get)
    t = ipp.Batch(frames, lanes=tbest, cfg=cfg, max_src=65536, mode="table")
    table_ms = timed(lambda: t.run(gs), gs)
    t.capture(gs)
    table_graph_ms = timed(lambda: t.launch(gs), gs)
    table_ws_gb = t.ws.numel() / 1e9
    t.close()
    del t
    mpix = sum(f.numel() for f in frames) / 1e6
    # the batched figure is the faster of the two forms, each as a graph
    table_wins = table_graph_ms < streams_graph_ms
    bat_ms = min(table_graph_ms, streams_graph_ms)
    return {"frames": n_frames, "mpix": mpix, "per_frame_ms": per_ms, "batched_ms": bat_ms,
            "form": ("table (one launch per stage over a device table of each lane's frames)" if table_wins
                     else "streams (per-frame launches over the lanes)") + ", captured graph",
            "speedup": per_ms / bat_ms, "batched_mpix_per_s": mpix / (bat_ms / 1e3),
            "table_ms": table_ms, "table_graph_ms": table_graph_ms, "table_workspace_gb": table_ws_gb,
            "table_lanes": tbest, "table_ms_lanes_1_2_4_8": [table_lane_ms[k] for k in (1, 2, 4, 8)],
            "streams_ms": streams_ms, "streams_graph_ms": streams_graph_ms, "lanes": best,
            "table_vs_streams": min(streams_ms, streams_graph_ms) / min(table_ms, table_graph_ms),
            "autotune_ms_lanes_1_2_4_8": lane_ms,
            "workload": f"{n_frames} frames of {sorted(set(shapes))}, {2000 * star_scale:g}-{50000 * star_scale:g} "
                        "stars, sky 200-3000 ADU, "
                        f"mesh {mesh}; per-frame ipp_extract on one stream, the stream form at its autotuned "
                        "lane count, and the table form"}


def raw_stream_leg(ipp, synth, dev, n_steps, n_resident=4):
    """Raw uint16 4096^2 frames (bias 500 ADU, radial flat 1.1 - 0.2 (r/r_max)^2,
    8,000 stars on a 1000 +- 50 ADU sky) resident on the device, streamed
    through bias/flat correction fused into the first reads, the catalog path,
    15 x 15 stamp cuts at the measured positions and the batched PSF fit of every
    catalog row; the row count stays on the device (no host round trip per
    frame).  Reports frames/s and sources/s."""
    import numpy as np
    import torch
    W = H = 4096
    yy, xx = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float64),
                            torch.arange(W, device=dev, dtype=torch.float64), indexing="ij")
    r = torch.hypot(xx - (W - 1) / 2.0, yy - (H - 1) / 2.0)
    flat = (1.1 - 0.2 * (r / r.max()) ** 2).float()
    inv_flat = (1.0 / flat.double()).float()
    raws = []
    for i in range(n_resident):
        scene = synth.frame_field_device(W, H, 8000, 5000 + i, device=dev).double()
        raw = torch.clamp(torch.round(500.0 + flat.double() * scene), 0, 65535).to(torch.int32)
        raws.append(raw.to(torch.int16))  # the uint16 bit pattern
    del yy, xx, r
    cfg = ipp.BgConfig(mesh=128)
    ex = ipp.Extractor(W, H, cfg, device=dev, max_src=65536)
    calib = (inv_flat, 500.0)

    nsrc_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    fit_out = {}

    def step(k):
        # the catalog count stays on the device: stamp cut and fit take it from there
        o = ex(raws[k % n_resident], calib=calib)
        st = ipp.stamp_cut(o["sub"], o["x"], o["y"], n_src=o["n_src"], S=15, max_src=ex.max_src)
        fit = ipp.psf_fit(st["stamps"], weights=st["weights"], n_src=o["n_src"], out=fit_out.get("o"))
        fit_out["o"] = fit
        nsrc_dev.add_(o["n_src"].clamp(max=ex.max_src))

    for k in range(2):
        step(k)
    torch.cuda.synchronize(dev)
    nsrc_dev.zero_()
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(n_steps):
        step(k)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    nsrc = int(nsrc_dev.item())
    return {"frames": n_steps, "frames_per_s": n_steps / (ms / 1e3), "sources_per_s": nsrc / (ms / 1e3),
            "ms_per_frame": ms / n_steps, "sources_per_frame": nsrc / max(n_steps, 1),
            "workload": "raw uint16 4096^2, bias 500, radial flat 0.9-1.1, 8,000 stars; calibration + catalog + "
                        "15x15 stamp cut + Moffat PSF fit of every catalog row, on one stream, counts on the device"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--psf-stamps", type=int, default=200000)
    ap.add_argument("--batch-frames", type=int, default=64)
    ap.add_argument("--raw-frames", type=int, default=10)
    ap.add_argument("--lanes", type=int, default=8, help="CUDA streams that consecutive frames rotate over")
    ap.add_argument("--soak-steps", type=int, default=3000,
                    help="steps run under the clock sampler before the timed ones (>= 1 s)")
    ap.add_argument("--cfg1-steps", type=int, default=200, help="1024^2 frames of the small-field line")
    args = ap.parse_args()
    ws, rank, local = dist_init()

    if args.impl == "reference":
        if rank != 0:
            return
        r = cpu_reference(args.steps, args.warmup)
        line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": "Mpix/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * r["sec"] / max(args.steps, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD},
                "cpu_baseline": {"value": r["value"], "unit": "Mpix/s", "cores": r["cores"], "kind": "oracle",
                                 "sample": r["sample"], "sources_per_s": r["sources_per_s"]},
                "e2e": {"value": r["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch

    import paper_2502_10783_gb300 as ipp
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ipp.load()

    img, truth = synth.frame_survey_4k(seed=1002 + rank)
    frames = [torch.from_numpy(img).to(dev) for _ in range(3)]
    cfg = ipp.BgConfig(mesh=MESH)
    ex = ipp.Extractor(W, H, cfg, device=dev, max_src=65536)
    stream = torch.cuda.current_stream(dev)
    # frames are independent: consecutive frames go round-robin to `lanes`
    # CUDA streams (one Extractor each), so that the latency-bound kernels of
    # one frame overlap those of the next; forked from and joined back to the
    # timing stream
    L = max(1, args.lanes)
    lane_st = [torch.cuda.Stream(dev) for _ in range(L)]
    lane_ex = [ex] + [ipp.Extractor(W, H, cfg, device=dev, max_src=65536) for _ in range(L - 1)]
    fork, joins = torch.cuda.Event(), [torch.cuda.Event() for _ in range(L)]

    def run_steps(n, body):
        fork.record(stream)
        for st in lane_st:
            st.wait_event(fork)
        for k in range(n):
            with torch.cuda.stream(lane_st[k % L]):
                body(k, k % L)
        for ln in range(L):
            joins[ln].record(lane_st[ln])
            stream.wait_event(joins[ln])

    def step(k, ln):
        lane_ex[ln](frames[k % 3], stream=lane_st[ln])

    run_steps(max(args.warmup, 3), step)
    torch.cuda.synchronize(dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-resident timed region ----------------------------------------
    # The clock sampler runs from a soak of >= 1 s of the same steps (timed too,
    # reported as `soak`) straight into the K timed steps, so that the clocks
    # and throttle reasons cover the timed region at steady state.
    soak_n = max(args.soak_steps, 0)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        s0.record(stream)
        run_steps(soak_n, step)
        s1.record(stream)
        e0.record(stream)
        run_steps(args.steps, step)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    soak = None
    if soak_n:
        sms = max_over_ranks(s0.elapsed_time(s1), ws, dev)
        soak = {"steps": soak_n, "ms": sms, "mpix_per_s": whole_job_rate(W * H / 1e6, soak_n, ws, sms)}
    K = int(ex.out["n_src"].item())
    mpix_step = W * H / 1e6
    value = whole_job_rate(mpix_step, args.steps, ws, ms)
    src_per_s = whole_job_rate(K, args.steps, ws, ms)

    # ---- end to end through the public API: pinned host frame in, catalog out -
    # Every step copies its frame from pinned host memory, runs the catalog
    # path and reads its catalog back, all on its lane's stream; the lanes
    # overlap one another's copies and kernels.
    host_in = torch.from_numpy(img).pin_memory()
    nmax = ex.max_src
    host_out = [{k: torch.empty(nmax, dtype=torch.float32).pin_memory() for k in ("x", "y", "flux")}
                for _ in range(L)]
    host_n = [torch.empty(1, dtype=torch.int32).pin_memory() for _ in range(L)]
    dframes = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(L)]

    def e2e_step(k, ln):
        dframes[ln].copy_(host_in, non_blocking=True)
        o = lane_ex[ln](dframes[ln], stream=lane_st[ln])
        host_n[ln].copy_(o["n_src"], non_blocking=True)
        for key in host_out[ln]:
            host_out[ln][key].copy_(o[key], non_blocking=True)

    run_steps(3, e2e_step)
    torch.cuda.synchronize(dev)
    n_e2e = max(50, args.steps)
    barrier()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    run_steps(n_e2e, e2e_step)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = max_over_ranks(a0.elapsed_time(a1), ws, dev)
    e2e_val = whole_job_rate(mpix_step, n_e2e, ws, ms_e2e)

    # ---- the 1024^2 gradient field (mesh 64): the small configuration ---------
    cfg1 = None
    if args.cfg1_steps > 0:
        img1, _ = synth.frame_gradient_1k(1001)
        f1 = [torch.from_numpy(img1).to(dev) for _ in range(3)]
        ex1 = [ipp.Extractor(1024, 1024, ipp.BgConfig(mesh=64), device=dev) for _ in range(L)]

        def step1(k, ln):
            ex1[ln](f1[k % 3], stream=lane_st[ln])

        run_steps(5, step1)
        torch.cuda.synchronize(dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        run_steps(args.cfg1_steps, step1)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        ms1 = max_over_ranks(c0.elapsed_time(c1), ws, dev)
        k1 = int(ex1[0].out["n_src"].item())
        cfg1 = {"workload": "gradient_1k: 1024x1024 float32, 1000 +- 50 ADU sky, 500 stars FWHM 3; mesh 64, 3x3 "
                            "filter, k=1.5, min_area 5, r=5, annulus 8-12 (fits in L2: 3 rotating 4 MiB frames)",
                "steps": args.cfg1_steps, "ms_per_step": ms1 / args.cfg1_steps,
                "mpix_per_s": whole_job_rate(1024 * 1024 / 1e6, args.cfg1_steps, ws, ms1),
                "sources_per_s": whole_job_rate(k1, args.cfg1_steps, ws, ms1), "sources_per_frame": k1}
        del f1, ex1

    # ---- per-stage breakdown (separate calls, CUDA events on this stream) ------
    stages = {}

    def timeit(fn, n=10):
        for _ in range(2):
            fn(0)
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for k in range(n):
            fn(k)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        return s0.elapsed_time(s1) / n

    bgws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    stages["bg_estimate"] = timeit(lambda k: ipp.bg_estimate(frames[k % 3], cfg=cfg, ws=bgws))
    mb, mr = ipp.bg_estimate(frames[0], cfg=cfg)
    subbuf = torch.empty((H, W), dtype=torch.float32, device=dev)
    stages["bg_subtract"] = timeit(lambda k: ipp.bg_subtract(frames[k % 3], mb, cfg=cfg, out=subbuf))
    dws = torch.empty(ipp.load().ipp_detect_label_workspace_size(W, H), dtype=torch.uint8, device=dev)
    stages["detect_label"] = timeit(lambda k: ipp.detect_label(subbuf, mr, cfg=cfg, max_src=65536, ws=dws))
    # detection on the pyramid-smoothed frame (the detection filter; a widening)
    stages["detect_label_filtered"] = timeit(
        lambda k: ipp.detect_label(subbuf, mr, cfg=cfg, max_src=65536, ws=dws, filter=1))
    lab, nsrc, st = ipp.detect_label(subbuf, mr, cfg=cfg, max_src=65536, ws=dws)
    stages["centroid"] = timeit(lambda k: ipp.centroid(subbuf, st["xbar"], st["ybar"], n_src=nsrc, max_src=65536))
    cx, cy, _, _ = ipp.centroid(subbuf, st["xbar"], st["ybar"], n_src=nsrc, max_src=65536)
    stages["aperture_phot"] = timeit(lambda k: ipp.aperture_phot(subbuf, cx, cy, n_src=nsrc, max_src=65536))
    # auto (Kron) photometry of the same catalog: a widening of the path, timed
    # beside it, not part of the step
    stages["auto_phot"] = timeit(lambda k: ipp.auto_phot(subbuf, lab, nsrc, st, max_src=65536))
    # deblending of the same candidates (also a widening, timed beside the step)
    dbws = torch.empty(ipp.load().ipp_deblend_workspace_size(W, H, 65536), dtype=torch.uint8, device=dev)
    stages["deblend"] = timeit(lambda k: ipp.deblend(subbuf, lab, nsrc, st, max_src=65536, ws=dbws))
    d_map, n_deb = ipp.deblend(subbuf, lab, nsrc, st, max_src=65536, ws=dbws)
    deblended_objects = int(n_deb.item())
    # cleaning of the deblended objects against the detection threshold (a
    # widening, timed beside the step)
    clws = torch.empty(ipp.load().ipp_clean_workspace_size(65536), dtype=torch.uint8, device=dev)
    stages["clean"] = timeit(lambda k: ipp.clean(subbuf, d_map, n_deb, 65536, mesh_rms=mr, cfg=cfg, ws=clws))
    cleaned_objects = int(ipp.clean(subbuf, d_map, n_deb, 65536, mesh_rms=mr, cfg=cfg, ws=clws)[1].item())
    # the natural-spline background map in place of the Keys cubic (a widening)
    spbuf = torch.empty_like(subbuf)
    stages["bg_subtract_spline"] = timeit(lambda k: ipp.bg_subtract_spline(frames[k % 3], mb, cfg=cfg, out=spbuf))
    del spbuf
    # the whole catalog path with the spline reading (interp = spline)
    cfg_sp = ipp.BgConfig(mesh=cfg.mesh, interp="spline")
    ex_sp = ipp.Extractor(W, H, cfg_sp, device=dev, max_src=65536)
    stages["extract_spline"] = timeit(lambda k: ex_sp(frames[k % 3]))
    del ex_sp
    # gray-scale maps of the subtracted frame (a widening, timed beside the step):
    # four distinct input/output pairs rotate, 512 MiB in all, so that each call
    # reads its input from HBM, not L2
    gin = [subbuf.clone() for _ in range(4)]
    gout = [torch.empty_like(subbuf) for _ in range(4)]
    gws = torch.empty(ipp.load().ipp_hist_equalize_workspace_size(4096), dtype=torch.uint8, device=dev)
    stages["gray_log"] = timeit(
        lambda k: ipp.gray_transform(gin[k % 4], ipp.GRAY_LOG, 0.0, 2000.0, a=1000.0, out=gout[k % 4]))
    stages["hist_equalize"] = timeit(lambda k: ipp.hist_equalize(gin[k % 4], nbins=4096, out=gout[k % 4], ws=gws))
    # zscale display limits of the same frames (1000 samples, one block)
    stages["zscale"] = timeit(lambda k: ipp.zscale(gin[k % 4]))
    # convolution and difference of image subtraction (49 basis kernels of 21 x 21,
    # spatial order 2, background order 1): the frame against a copy of itself
    # as the template, fixed coefficients (the fit is not part of this call)
    sub_coef = np.zeros(49 * 6 + 3, np.float32)
    sub_coef[0] = 1.0 / (2.0 * np.pi * 0.7 ** 2)
    sub_coef = torch.from_numpy(sub_coef).to(dev)      # resident: no copy inside the timed calls
    sub_ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    stages["sub_apply"] = timeit(
        lambda k: ipp.sub_apply(gin[k % 4], gin[(k + 1) % 4], sub_coef, out=gout[k % 4], ws=sub_ws))
    # the fit of the same pair: 10 x 10 regions, 21 x 21 footprints, FP64 normal
    # equations of the 49-function basis (297 unknowns) and their Cholesky solve
    fit_ws = torch.empty(ipp.load().ipp_sub_fit_workspace_size(
        100, 100, 10, 10, 3, np.array([6, 4, 2], np.int32).ctypes.data_as(ctypes.c_void_p), 2, 1),
        dtype=torch.uint8, device=dev)
    stages["sub_fit"] = timeit(lambda k: ipp.sub_fit(gin[k % 4], gin[(k + 1) % 4], ws=fit_ws), n=5)
    sub_fit_status = int(ipp.sub_fit(gin[0], gin[1], ws=fit_ws)["status"].item())
    # image alignment of the subtracted frame onto a second exposure's pixel grid
    # (a widening): WCS mapping of a 32 px node grid, partial affine fit, bilinear
    # reprojection; same four rotating input/output pairs
    src_wcs, tgt_wcs = synth.wcs_pair(W, H, seed=7300)
    stages["align"] = timeit(lambda k: ipp.align(gin[k % 4], src_wcs, tgt_wcs, W, H, step=32, out=gout[k % 4]))
    xo_, yo_ = ipp.wcs_map(src_wcs, tgt_wcs, W, H, step=32)
    Maff, _ = ipp.affine_fit(xo_, yo_, grid_step=32)
    Mi_ = Maff[6:].clone()
    stages["reproject"] = timeit(lambda k: ipp.reproject_affine(gin[k % 4], Mi_, W, H, out=gout[k % 4]))
    del gin, gout

    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    # dominant memory-bound kernel of the step: mesh statistics (one read of the frame)
    bg_ms = stages["bg_estimate"]
    roof = {"kernel": "k_mesh_stats (+ the 32x32 k_mesh_filter: one ipp_bg_estimate call)", "bound": "hbm",
            "achieved": W * H * 4 / (bg_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "traffic": profiled_traffic("paper_2502_10783_gb300/csrc/bg.cu", "profiles/k_mesh_stats.survey_4k.md"),
            "algorithmic_bytes": W * H * 4,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in pk else "fallback"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    step_ms = ms / args.steps
    whole = {"algorithmic_bytes_per_step": 16 * W * H, "achieved_gbs": 16 * W * H / (step_ms / 1e3) / 1e9}
    whole["frac_of_measured_hbm"] = whole["achieved_gbs"] / hbm
    whole["frac_of_nominal_hbm"] = whole["achieved_gbs"] / 7900.0
    # gray maps: the log map reads and writes each pixel once (8 B/px); equalisation
    # reads the frame three times (min/max, histogram, apply) and writes it once
    # (16 B/px; 12 B/px would be the floor of any two-pass form)
    gray = {}
    for key, bpp, kern in (("gray_log", 8, "k_gray"), ("hist_equalize", 16, "k_minmax + k_hist + k_cdf + k_equalize")):
        gb = bpp * W * H / (stages[key] / 1e3) / 1e9
        gray[key] = {"kernels": kern, "bytes_per_px": bpp, "ms": stages[key], "achieved_gbs": gb,
                     "frac_of_measured_hbm": gb / hbm}
    # image subtraction: 441 taps a pixel (2 flops each) plus the tile kernels
    # (49 x 441 multiply-adds a tile); FP32 ALU-bound
    sub_flops = 2.0 * 441 * W * H + 2.0 * 49 * 441 * ((W + 20) // 21) * ((H + 20) // 21)
    subtraction = {"ms": stages["sub_apply"], "achieved_tflops": sub_flops / (stages["sub_apply"] / 1e3) / 1e12,
                   "flops_per_call": sub_flops, "kernels": "k_sub_basis + k_sub_apply (one block per 21 x 21 tile)",
                   "workload": "survey_4k subtracted frame against a copy, 21 x 21 kernel, 49 basis functions",
                   "fit_ms": stages["sub_fit"], "fit_status": sub_fit_status,
                   "fit_kernels": "k_sub_stamps + k_sub_compact + k_sub_conv + k_sub_gram + k_sub_assemble + "
                                  "blocked Cholesky k_chol_diag / k_chol_trsm / k_chol_syrk per 32-column panel + "
                                  "k_chol_solve (FP64; 10 x 10 regions, 297 unknowns)"}
    gb = 8 * W * H / (stages["reproject"] / 1e3) / 1e9
    align = {"ms": stages["align"], "reproject_ms": stages["reproject"], "reproject_bytes_per_px": 8,
             "reproject_achieved_gbs": gb, "reproject_frac_of_measured_hbm": gb / hbm,
             "kernels": "k_wcs_map (32 px nodes, FP64) + k_aff_sum1/2 + k_aff_solve + k_reproject",
             "workload": "survey_4k subtracted frame onto a second exposure's grid (pointing offset "
                         "0.02-0.05 deg, rotated, SIP order 3 on both)"}

    # ---- PSF fit leg: 200k Moffat stamps ---------------------------------------
    psf = None
    if args.psf_stamps > 0:
        stamps, _ = synth.moffat_stamps(args.psf_stamps, seed=4000, oversample=3)
        ts = torch.from_numpy(stamps).to(dev)
        ipp.psf_fit(ts[:1000])
        torch.cuda.synchronize(dev)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        fit = ipp.psf_fit(ts)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pms = p0.elapsed_time(p1)
        it = fit["iters"].float().mean().item()
        conv = (fit["flags"] == 0).float().mean().item()
        psf = {"stamps_per_s": args.psf_stamps / (pms / 1e3), "ms": pms, "n": args.psf_stamps,
               "mean_iters": it, "converged_frac": conv,
               "converged_stamps_per_s": conv * args.psf_stamps / (pms / 1e3),
               "stop_rule": "Gauss-Newton decrease <= 1e-10 chi^2 + 1e-12 sum (m - sky)^2, or lambda > 1e10; "
                            "max_iter 50 (faint stamps that crawl are flagged FIT_MAXITER)",
               "workload": "200,000 15x15 elliptical Moffat stamps (beta 2.5), 7-parameter LM, FP64 solve",
               "kernel": "k_psf_fit (one stamp per lane, 32 per warp)"}
        psf_stamps_host = stamps

    # ---- raw uint16 stream: calibration through PSF fit ------------------------
    raw = None
    if args.raw_frames > 0:
        raw = raw_stream_leg(ipp, synth, dev, args.raw_frames)

    # ---- batched leg: frames of mixed sizes, per-frame calls vs the batch graph -
    batch = None
    if args.batch_frames > 0:
        batch = batch_leg(ipp, synth, dev, args.batch_frames)
        # many small frames: the launch-bound case the table form is for
        batch["small_frames"] = batch_leg(ipp, synth, dev, args.batch_frames,
                                          shapes=[(1024, 1024)] * args.batch_frames, mesh=64,
                                          star_scale=1.0 / 16)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        single = cpu_single_core(img)          # plain build first: use_openmp switches the process
        n_cpu = 1000
        t0 = time.perf_counter()
        if psf is not None:
            oracle.psf_fit(psf_stamps_host[:n_cpu])
        dt1 = time.perf_counter() - t0
        cores = oracle_all_cores()
        r = cpu_reference(steps=2, warmup=0, img=img, cores=cores)
        cpu = {"value": r["value"], "unit": "Mpix/s", "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
               "sources_per_s": r["sources_per_s"], "single_core": single}
        if psf is not None:
            n_all = 4000
            t0 = time.perf_counter()
            oracle.psf_fit(psf_stamps_host[:n_all])
            dt = time.perf_counter() - t0
            psf["cpu_baseline"] = {"value": n_all / dt, "unit": "stamps/s", "cores": cores, "kind": "oracle",
                                   "sample": f"the first {n_all} of the same stamps, OpenMP build",
                                   "single_core": {"value": n_cpu / dt1, "unit": "stamps/s", "cores": 1,
                                                   "sample": f"the first {n_cpu} stamps, plain build"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "parallelism": f"replicas x{ws} (independent frames), {L} streams per GPU",
                       "l2": "inputs larger than L2: 3 rotating 64 MiB frames"},
            "sources_per_s": src_per_s, "sources_per_frame": K, "deblended_objects_per_frame": deblended_objects,
            "cleaned_objects_per_frame": cleaned_objects,
            "e2e": {"value": e2e_val, "unit": "Mpix/s", "h2d_bytes_per_step": W * H * 4,
                    "pipelining": f"each step H2D + catalog + D2H on one of {L} lane streams",
                    "d2h_bytes_per_step": 4 + 3 * 4 * nmax},
            "gpu_launches": KERNELS_PER_FRAME * args.steps,
            "roofline": roof, "step_roofline": whole, "stages_ms": stages, "gray_maps": gray, "alignment": align, "subtraction": subtraction,
            "clocks": clk.summary(), "soak": soak, "cfg1_1k": cfg1, "psf_fit": psf, "batched": batch,
            "raw_u16_stream": raw,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

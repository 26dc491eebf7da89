"""Benchmark of the layered Gaussian-splatting rasterizer on GB300.

One step = one pass of the whole hot path over the 1.2M-Gaussian layered
CT-like scene (5 nested shells, SH degree 3, 1024x1024, random 5-bit layer
mask, one clip plane): S1 preprocess, S2 depth radix sort + tile binning, S3
compositing, S4 backward (with per-Gaussian contributions) and S5 prune.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

After the timed steps (rank 0, N = 1) a serving leg replays 512 Poisson
requests at 300/s against three resident models (0.5M, 1.5M, 3M Gaussians)
through the served path (continuous batching into batched launches) and the
plain path (one request at a time), in real time and saturated; its p50/p99
latencies and Mpixels/s go under "serving".

Prints one JSON line.  The reference arm times the FP64 CPU oracle on a
bounded sample of the same workload (this method has no runnable reference
implementation).  Multi-GPU runs (torchrun) are independent replicas: the
path has no exchange step, every rank renders the full frame.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixels/s & p50/p99 frame ms (served vs plain) at PSNR>=50dB vs FP64 oracle"
UNIT = "Mpixels/s"
WORKLOAD = ("layered CT-like scene: 1.2M Gaussians in 5 layers (400k/300k/250k/100k/150k shells), SH degree 3, "
            "1024x1024, random 5-bit layer mask + 1 clip plane; step = forward + backward + contribution prune")
# Per-pair arithmetic of the compositor kernels (FLOPs, an FMA counts 2).  A pair
# is (pixel, list entry) up to the pixel's n_contrib.  The roofline uses the
# scope table's per-pair figures for every such pair: about 20 FLOP for the
# forward (alpha and blend) and 2.5 times that for the backward.
# roofline_detail and roofline_all count the evaluation of every pair and the
# blend arithmetic only for the pairs that were blended (the status word's
# n_blended).
FLOP_S3_PAIR = 20      # forward compositing per evaluated pair
FLOP_S4_PAIR = 50      # backward compositing per evaluated pair (2.5 x forward)
FLOP_EVAL = 14         # alpha of one pair: offsets, exponent, exp2, opacity, clamp, threshold test
FLOP_BLEND_FWD = 10    # blending a splat into a pixel
FLOP_BLEND_BWD = 40    # gradient of one blended pair


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# DRAM bytes per step of each stage (dram__bytes_read.sum + dram__bytes_write.sum
# over the stage's kernels) from one ncu capture of this workload (the launch
# list summarised in profiles/c2_step_launch_list.md; ncu flushes the caches
# before every kernel, so these are cold-cache bytes).  A figure is reported
# only while the source file of the stage's kernels is byte-identical to the
# one profiled.
_CSRC = "paper_2410_16978_gb300/csrc/"
_SHA = {"preprocess.cu": "eb1b766eb81eb63ee835a4bc6dbec6025330022db2616323c04256d968baad77",
        "sort.cu": "e150c0bf91f5999fb2aa087435f6814b59e87827a3e158c55ec96cf51630142d",
        "bin.cu": "7cedc04ab2c91de8c398824e382a72c0011f1e2d1510aba0fac2598cced73bcb",
        "composite.cu": "e565523be6ac5bd421de1f94cfeeaf10e25dd7b0246be515cc9dc6f9d6651788",
        "preprocess_bwd.cu": "770f5bae4d75d26337f17e9c0c8194b9317d4b3449043b4bf36999300b41d3d1"}
PROFILED_TRAFFIC = {   # stage: (bytes per step, source file, kernels)
    "preprocess": (165798637, "preprocess.cu", "k_preprocess"),
    "compact": (7833965, "sort.cu", "k_sort_hist"),
    "depth_sort": (14909696, "sort.cu", "k_sort_pass x4"),
    "bin_rows": (68223268, "bin.cu", "k_bin_rows x2, k_bin_rowscan"),
    "bin_tiles": (25201133, "bin.cu", "k_bin_tiles x2, k_bin_tiles_scan"),
    "composite": (36194176, "composite.cu", "k_composite_fwd"),
    "composite_bwd": (72336974, "composite.cu", "k_composite_bwd"),
    "preprocess_bwd": (448030148, "preprocess_bwd.cu", "k_preprocess_bwd"),
    "prune": (9623217, "sort.cu", "k_scan_reduce, k_scan_down"),
}


def profiled_traffic(stage: str):
    import hashlib
    rec = PROFILED_TRAFFIC.get(stage)
    if not rec:
        return None
    with open(os.path.join(ROOT, _CSRC + rec[1]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != _SHA[rec[1]]:
            return None
    return rec[0]


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (every rank gets it)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(pixels_per_step: int, steps: int, world: int, total_ms: float) -> float:
    """Pixels of all replicas / the max-over-ranks time, in Mpixels/s."""
    return world * pixels_per_step * steps / (total_ms / 1e3) / 1e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def build_workload():
    import synth
    w = synth.scene_c2()
    return w


# ----------------------------------------------------------------------------- oracle (CPU) timing

def host_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))


def _oracle_map(fn, items, threads):
    """fn over items on `threads` host threads (the oracle's C functions run
    without the Python lock, so the threads run on separate cores)."""
    if threads <= 1:
        return [fn(x) for x in items]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, items))


def _chunks(n, parts):
    step = -(-n // max(1, parts))
    return [slice(a, min(n, a + step)) for a in range(0, n, step)]


def oracle_preprocess(sc, cam, mask, planes, threads):
    """FP64 preprocess of all Gaussians, split into contiguous chunks (each
    Gaussian is independent)."""
    import oracle
    parts = _oracle_map(lambda sl: oracle.preprocess(sc.subset(sl), cam, mask, planes, "f64"),
                        _chunks(sc.n, 4 * threads), threads)
    pre = {k: np.concatenate([p[k] for p in parts]) for k in parts[0] if isinstance(parts[0][k], np.ndarray)}
    pre["W"], pre["H"] = int(cam.width), int(cam.height)
    return pre


def _row_bands(H, bands):
    """Tile rows dealt round-robin into `bands` sets (so each set mixes heavy
    central rows and light edge rows)."""
    Ty = (H + 15) // 16
    return [np.arange(k, Ty, bands) for k in range(min(bands, Ty))]


def oracle_forward(pre, ranges, lst, bg, threads):
    """FP64 compositing of every pixel, tile rows spread over the threads."""
    import oracle
    W, H = pre["W"], pre["H"]
    img = np.zeros((3, H, W))
    alpha = np.zeros((H, W))
    info = {"fragile": 0, "multi_fragile": 0}

    def band(rows):
        ys = np.concatenate([np.arange(r * 16, min(H, r * 16 + 16)) for r in rows])
        gy, gx = np.meshgrid(ys, np.arange(W), indexing="ij")
        cp = oracle.composite_pixels(pre, ranges, lst, gx.ravel(), gy.ravel(), bg)
        return gx.ravel(), gy.ravel(), cp

    for xs, ys, cp in _oracle_map(band, _row_bands(H, 4 * threads), threads):
        img[:, ys, xs] = cp["rgb"].T
        alpha[ys, xs] = cp["alpha"]
        info["fragile"] += int((cp["fragile"] > 0).sum())
        info["multi_fragile"] += int((cp["fragile"] > 1).sum())
    return img, alpha, info


def oracle_backward(pre, ranges, lst, bg, dimg, dal, threads):
    """FP64 compositing backward over every pixel: each thread takes a set of
    tile rows; record gradients and blend weights add up (the max for
    contrib_max) over the sets."""
    import oracle
    W, H = pre["W"], pre["H"]
    Tx = (W + 15) // 16

    def band(rows):
        tm = np.zeros(len(ranges), np.uint8)
        for r in rows:
            tm[r * Tx:(r + 1) * Tx] = 1
        return oracle.composite_backward(pre, ranges, lst, bg, dimg, dal, tm)

    out = None
    for cb in _oracle_map(band, _row_bands(H, threads), threads):
        if out is None:
            out = dict(rec_grad=cb["rec_grad"].copy(), contrib_sum=cb["contrib_sum"].copy(),
                       contrib_max=cb["contrib_max"].copy())
        else:
            out["rec_grad"] += cb["rec_grad"]
            out["contrib_sum"] += cb["contrib_sum"]
            np.maximum(out["contrib_max"], cb["contrib_max"], out=out["contrib_max"])
    return out


def oracle_chain(sc, cam, vis, rec_grad, threads):
    import oracle
    parts = _oracle_map(lambda sl: oracle.chain(sc.subset(sl), cam, vis[sl], rec_grad[sl]),
                        _chunks(sc.n, 4 * threads), threads)
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def oracle_step(w, dimg, dal, threads, backward=True):
    """One pass of the hot path on the FP64 oracle over the whole frame:
    preprocess, binning, compositing of every pixel, and (backward=True) the
    compositing backward of every pixel, the chain rule and the prune.
    Returns (seconds per stage, image, detail)."""
    import oracle
    oracle.build()
    sc, cam = w["scene"], w["cameras"][0]
    bg = tuple(float(v) for v in w["bg"])
    t = [time.perf_counter()]
    pre = oracle_preprocess(sc, cam, w["layer_mask"], w["planes"], threads)
    t.append(time.perf_counter())
    ranges, lst = oracle.bin_tiles(pre)
    t.append(time.perf_counter())
    img, alpha, info = oracle_forward(pre, ranges, lst, bg, threads)
    t.append(time.perf_counter())
    names = ["preprocess", "binning", "forward"]
    if backward:
        cb = oracle_backward(pre, ranges, lst, bg, dimg, dal, threads)
        t.append(time.perf_counter())
        oracle_chain(sc, cam, pre["vis"], cb["rec_grad"], threads)
        t.append(time.perf_counter())
        oracle.prune(cb["contrib_max"], 0.005)
        t.append(time.perf_counter())
        names += ["backward", "chain", "prune"]
    stages = {k: t[i + 1] - t[i] for i, k in enumerate(names)}
    info.update(visible=int(pre["vis"].sum()), pairs=int(lst.shape[0]))
    return stages, img, info


def _workload_config(w, world):
    """The `config` object of both arms (the workload, nothing about the implementation)."""
    sc, cam = w["scene"], w["cameras"][0]
    scene_mb = sum(a.nbytes for a in (sc.means, sc.log_scales, sc.quats, sc.opacity_logit, sc.sh)) / 1e6
    return {"workload": WORKLOAD, "gaussians": sc.n, "width": cam.width, "height": cam.height,
            "l2": "inputs larger than L2 (scene %.0f MB)" % scene_mb,
            "parallelism": "replicas x%d" % world if world > 1 else "single device"}


def _upstream_grads(W, H):
    rng = np.random.default_rng(7)
    dimg = rng.standard_normal((3, H, W)).astype(np.float32) / (3 * W * H)
    dal = rng.standard_normal((H, W)).astype(np.float32) / (W * H)
    return dimg, dal


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is the whole c2 step (full
    frame, forward + backward + prune) in FP64 on all host cores; its measured
    wall time is the step time."""
    if rank != 0:
        return
    w = build_workload()
    cam = w["cameras"][0]
    threads = host_threads()
    dimg, dal = _upstream_grads(cam.width, cam.height)
    for _ in range(args.warmup):
        oracle_step(w, dimg, dal, threads)
    walls, stage_sum, info = [], {}, None
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        stages, _, info = oracle_step(w, dimg, dal, threads)
        walls.append(time.perf_counter() - t0)
        for k, v in stages.items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    ms = 1e3 * statistics.mean(walls)
    v = cam.width * cam.height / (ms / 1e3) / 1e6
    sample = ("the whole step on the full %dx%d frame: FP64 preprocess of all %d Gaussians, binning, compositing "
              "and compositing backward of every pixel, chain rule, prune; %d host threads over tile rows and "
              "Gaussian chunks" % (cam.width, cam.height, w["scene"].n, threads))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _workload_config(w, world),
            "mode": "FP64 CPU oracle (C), %d threads" % threads,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "stages_s_per_step": {k: round(x / len(walls), 4) for k, x in stage_sum.items()},
            "wall_s_min_max": [round(min(walls), 4), round(max(walls), 4)],
            "visible": info["visible"], "pairs": info["pairs"]}
    print(json.dumps(line), flush=True)


def oracle_baselines(w, gpu_image, threads):
    """The oracle timed beside the GPU (rank 0, N = 1): the whole c2 step on
    all host threads (full frame), with the PSNR of the GPU image against its
    FP64 image over every pixel; the 128x128 workload's full frame on one and
    on all threads; the forward of each eye of the 3M stereo workload
    (2064x2208) on all threads."""
    import synth
    cam = w["cameras"][0]
    dimg, dal = _upstream_grads(cam.width, cam.height)
    t0 = time.perf_counter()
    stages, img, info = oracle_step(w, dimg, dal, threads)
    wall = time.perf_counter() - t0
    mse = float(((gpu_image.astype(np.float64) - img) ** 2).mean())
    psnr = float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)
    err = np.abs(gpu_image.astype(np.float64) - img).max(0)
    w1 = synth.scene_c1()
    c1 = {}
    for th in (1, threads):
        t1 = time.perf_counter()
        oracle_step(w1, *_upstream_grads(128, 128), th, backward=False)
        c1["forward_ms_%d_thread%s" % (th, "s" if th > 1 else "")] = round(1e3 * (time.perf_counter() - t1), 3)
    w4 = synth.scene_c4()
    c4 = {}
    for eye, cam4 in zip(("left", "right"), w4["cameras"]):
        t1 = time.perf_counter()
        st4, _, inf4 = oracle_step(dict(w4, cameras=[cam4]), None, None, threads, backward=False)
        c4[eye] = {"forward_s": round(time.perf_counter() - t1, 3),
                   "stages_s": {k: round(v, 3) for k, v in st4.items()}, "pairs": inf4["pairs"]}
    detail = {"c2_step_s": round(wall, 4), "c2_stages_s": {k: round(v, 4) for k, v in stages.items()},
              "c1_full_frame": c1, "c4_eyes_full_frame": c4, "threads": threads}
    parity = {"psnr_db_full_frame": psnr, "max_abs_err": float(err.max()),
              "fragile_pixels": info["fragile"], "multi_fragile_pixels": info["multi_fragile"],
              "pixels": int(cam.width * cam.height)}
    return cam.width * cam.height / wall / 1e6, wall, detail, parity


# ----------------------------------------------------------------------------- GPU arm

SERVE_MODELS = (("0.5M", 0.5 / 1.2), ("1.5M", 1.25), ("3M", None))
SERVE_SIZES = ((512, 512, 1), (1024, 1024, 1), (2064, 2208, 2))


def per_view_forward(models, dev, renders=20, warmup=3):
    """Device time of one forward view of every serving model at every view
    size: one gs_render through the public Rasterizer (camera at
    (0.3, -0.2, 3.6) looking at the origin, every layer, no plane), recorded
    once as a CUDA graph and replayed, CUDA events over `renders` replays
    after `warmup` (workspace sized by a first, checked render).  The graph
    takes the host's launch overhead out, so this is the view's GPU time."""
    import synth
    import torch
    from paper_2410_16978_gb300 import Rasterizer

    out = {}
    for name, ds in models.items():
        row = {}
        for W, H, _ in SERVE_SIZES:
            cam = synth.look_at_camera((0.3, -0.2, 3.6), width=W, height=H)
            r = Rasterizer(ds.n, W, H, device=dev)
            img, al = r.render(ds, cam, check=True)
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):
                r.render(ds, cam, image=img, alpha=al, check=False)
            torch.cuda.current_stream(dev).wait_stream(side)
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                r.render(ds, cam, image=img, alpha=al, check=False)
            for _ in range(warmup):
                g.replay()
            st = torch.cuda.current_stream(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(st)
            for _ in range(renders):
                g.replay()
            e1.record(st)
            torch.cuda.synchronize(dev)
            if r.status().error != 0:
                raise RuntimeError("per-view render of %s %dx%d failed" % (name, W, H))
            row["%dx%d" % (W, H)] = round(e0.elapsed_time(e1) / renders, 4)
            del g, r, img, al
        out[name] = row
    return out


def run_serving(dev, n_requests=512, rate=300.0, budget=8 << 30, replays=3):
    """Three resident layered models (0.5M, 1.5M, 3M Gaussians, SH degree 3)
    and a Poisson trace of mixed requests, replayed in real time through the
    served path (continuous batching) and through the plain path (one request
    per gs_render sequence, FIFO), then replayed saturated (all requests at
    t = 0) for peak throughput.

    Both modes start every replay from the same calibration: the pair
    capacities are sized once (36 random views, then one saturated pass of
    the trace itself), and before each replay the capacities are restored,
    the buffer pools dropped and re-filled by a short warm-up in that mode.
    The 300 req/s trace is replayed `replays` times per mode in alternating
    order (plain, served, served, plain, ...); medians and ranges are
    reported with the retries of every replay.  One served request is
    rendered again and compared with the FP64 oracle."""
    import synth
    import torch
    from paper_2410_16978_gb300 import DeviceScene
    from paper_2410_16978_gb300.serve import RenderServer, make_trace, summarize

    models, hosts = {}, {}
    for name, scale in SERVE_MODELS:
        sc = synth.scene_c4()["scene"] if scale is None else synth.scene_c2(scale=scale)["scene"]
        hosts[name] = sc
        models[name] = DeviceScene.from_host(sc, device=dev)
    srv = RenderServer(models, memory_budget=budget, device=dev)
    rng = np.random.default_rng(synth.config_seed(5))
    cal = make_trace(np.random.default_rng(1), list(models), n_requests=36, rate=None, sizes=SERVE_SIZES)
    for req in cal:
        srv.calibrate(req.model, req.cameras, req.layer_mask, req.planes)
    trace = make_trace(rng, list(models), n_requests=n_requests, rate=rate, sizes=SERVE_SIZES)
    sat = [dataclasses.replace(r, arrival=0.0) for r in trace]
    srv.run_trace(sat, "served")                  # sizes the capacities of every (model, size) of the trace
    caps = srv.capacities()
    out = {"models": {k: m.n for k, m in models.items()}, "requests": n_requests, "rate_rps": rate,
           "memory_budget_gib": budget / 2 ** 30, "sizes": ["%dx%dx%d" % s for s in SERVE_SIZES],
           "mpixels_total": sum(r.pixels for r in trace) / 1e6, "replays_per_mode": replays,
           "calibration": "36 random views + one saturated served pass of the trace; restored before every replay"}

    def replay(tr, mode):
        srv.set_capacities(caps)
        srv.run_trace(sat[:64], mode)             # refills the pools in this mode
        r0, b0, v0 = srv.retries, srv.batches, srv.views_launched
        res, wall = srv.run_trace(tr, mode)
        s = summarize(res, tr, wall)
        s.update(retries=srv.retries - r0, launches=(srv.batches - b0) if mode == "served" else None,
                 views=srv.views_launched - v0)
        return s

    order = [("plain", "served")[(k // 2 + k) % 2] for k in range(2 * replays)]   # ABBAAB...
    runs = {"plain": [], "served": []}
    for mode in order:
        runs[mode].append(replay(trace, mode))
    for mode, rs in runs.items():
        med = {k: statistics.median(r[k] for r in rs) for k in ("mpix_s", "p50_ms", "p99_ms", "mean_ms")}
        med.update({k + "_range": [round(min(r[k] for r in rs), 4), round(max(r[k] for r in rs), 4)]
                    for k in ("mpix_s", "p50_ms", "p99_ms")})
        med["retries"] = [r["retries"] for r in rs]
        med["by_size_p50_p99_ms"] = rs[len(rs) // 2]["by_size_p50_p99_ms"]
        med["views"] = rs[0]["views"]
        if mode == "served":
            med["launches"] = [r["launches"] for r in rs]
        out["trace_%s" % mode] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in med.items()}
    for mode in ("plain", "served"):
        s = replay(sat, mode)
        out["saturated_%s" % mode] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()}
    out["order"] = order
    out["per_view_forward_ms"] = per_view_forward(models, dev)

    # one served request (a 1024x1024 view of the 1.5M model) against the FP64 oracle
    import oracle
    req = next(r for r in trace if r.model == "1.5M" and r.cameras[0].width == 1024)
    srv.set_capacities(caps)
    res, _ = srv.run_trace([dataclasses.replace(req, arrival=0.0)], "served", keep_images=True)
    torch.cuda.synchronize()
    img = res[0].images[0].cpu().numpy().astype(np.float64)
    cam = req.cameras[0]
    prng = np.random.default_rng(3)
    xs = prng.integers(0, cam.width, 16384).astype(np.int32)
    ys = prng.integers(0, cam.height, 16384).astype(np.int32)
    pre = oracle.preprocess(hosts[req.model], cam, req.layer_mask, req.planes, "f64")
    ranges, lst = oracle.bin_tiles(pre)
    cp = oracle.composite_pixels(pre, ranges, lst, xs, ys, req.bg)
    mse = float(((img[:, ys, xs].T - cp["rgb"]) ** 2).mean())
    out["served_view_psnr_db_vs_fp64_oracle"] = float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)
    out["served_view"] = "request %d: 1.5M model, 1024x1024, mask %d, %d plane(s); 16384 random pixels" % (
        req.rid, req.layer_mask, len(req.planes))
    return out


def run_training(dev, steps=24):
    """The training workload: 500k Gaussians in 3 shell layers (SH degree 3),
    8 cameras on a sphere of radius 4 at 800x800, targets rendered from the
    seeded perturbed copy of the scene.  One step = one view through the
    autograd Functions: render, 0.8 L1 + 0.2 D-SSIM + 0.8 alpha-L1 loss under
    a random background, backward with blend weights, Adam on every layer;
    after the timed steps one contribution prune at 0.005."""
    import torch
    import synth
    from paper_2410_16978_gb300 import DeviceScene, Rasterizer, gs_profile_collect, gs_profile_enable
    from paper_2410_16978_gb300.train import TrainConfig, Trainer

    w = synth.scene_c3()
    cams = w["cameras"]
    W, H = cams[0].width, cams[0].height
    tds = DeviceScene.from_host(w["target_scene"], device=dev)
    targets = []
    for cam in cams:
        r = Rasterizer(tds.n, W, H, device=dev)
        img, al = r.render(tds, cam, w["layer_mask"], (), (0.0, 0.0, 0.0), check=True)
        targets.append((img.clone(), al.clone()))
    del tds
    tr = Trainer(DeviceScene.from_host(w["scene"], device=dev), cams, TrainConfig(w_alpha=0.8))
    rng = np.random.default_rng(synth.config_seed(3))
    bgs = [tuple(float(v) for v in rng.uniform(0, 1, 3)) for _ in range(steps + 8)]
    for k in range(8):                                        # warm-up: one pass over the views
        tr.step(k % 8, *targets[k % 8], bgs[k])
    torch.cuda.synchronize()
    gs_profile_collect()
    gs_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    losses = []
    e0.record()
    for k in range(steps):
        losses.append(tr.step(k % 8, *targets[k % 8], bgs[8 + k]))
    e1.record()
    torch.cuda.synchronize()
    gs_profile_enable(False)
    prof = gs_profile_collect()
    ms = e0.elapsed_time(e1) / steps
    n0 = tr.scene.n
    n1 = tr.prune()
    return {"workload": "500k Gaussians, 3 layers, SH3, 8 views 800x800, Adam on all layers, random background",
            "steps": steps, "ms_per_step": round(ms, 4), "mpix_s": round(W * H / (ms / 1e3) / 1e6, 2),
            "loss_first": round(float(losses[0]), 6), "loss_last": round(float(losses[-1]), 6),
            "prune_threshold": 0.005, "gaussians_before_prune": n0, "gaussians_after_prune": n1,
            "stages_ms_per_step": {k: round(v[0] / steps, 4) for k, v in prof.items() if v[1]},
            "targets": "rendered on the GPU from the perturbed scene (the parity tests use oracle renders)"}


def run_stereo(dev, frames=20, warmup=3):
    """The mixed-precision stereo workload's frame (3M Gaussians, 2 x
    2064x2208, FP32 storage): gs_render_stereo with a depth sort per eye and
    with the shared-eye sort (paper Sec. 3.3), CUDA events over `frames`
    frames after `warmup`; the right eye of the shared sort against the exact
    right eye."""
    import torch
    import synth
    from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
    w = synth.scene_c4()
    sc, cams, mask, planes = w["scene"], w["cameras"], w["layer_mask"], w["planes"]
    bg = (0.0, 0.0, 0.0)
    ds = DeviceScene.from_host(sc, device=dev)
    rs = [Rasterizer(sc.n, c.width, c.height, device=dev) for c in cams]
    for r, c in zip(rs, cams):
        r.render(ds, c, mask, planes, bg, check=True)
        r._alloc(int(r.dup_capacity * 1.1) + 4096)      # the shared order adds the other eye's Gaussians
    imgs = [torch.empty((3, c.height, c.width), device=dev) for c in cams]
    als = [torch.empty((c.height, c.width), device=dev) for c in cams]
    cs, cl, cr = ds.c_struct(), _lib.make_camera(cams[0]), _lib.make_camera(cams[1])
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "3M Gaussians in 5 layers, SH3 FP32, stereo 2 x 2064x2208 (64 mm), frames of both eyes"}
    right = {}
    for shared in (False, True):
        def frame():
            _lib.gs_render_stereo(cs, cl, cr, mask, list(planes), bg, rs[0].workspace, rs[0].ws_bytes,
                                  rs[1].workspace, rs[1].ws_bytes, imgs[0], als[0], imgs[1], als[1], shared,
                                  int(stream.cuda_stream))
        for _ in range(warmup):
            frame()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
        for e0, e1 in ev:
            e0.record(stream)
            frame()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        assert rs[0].status().error == 0 and rs[1].status().error == 0
        right[shared] = imgs[1].clone()
        out["shared_sort" if shared else "per_eye_sort"] = {"ms_p50": round(ms[len(ms) // 2], 4),
                                                             "ms_min": round(ms[0], 4),
                                                             "mpix_s": round(2 * cams[0].width * cams[0].height /
                                                                             (ms[len(ms) // 2] / 1e3) / 1e6, 1)}
    d = (right[True] - right[False]).double()
    mse = float((d * d).mean())
    out["right_eye_psnr_shared_vs_per_eye_db"] = float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)
    out["right_eye_max_abs_diff"] = float(d.abs().max())
    out["speedup"] = round(out["per_eye_sort"]["ms_p50"] / out["shared_sort"]["ms_p50"], 4)
    return out


def stage_work(rast, sc, st, W, H):
    """Algorithmic bytes (or FLOPs) of each step of the hot path for the
    rendered frame, from the counts in its workspace: N Gaussians, V visible,
    R (Gaussian, tile row) entries, D (tile, Gaussian) pairs, the depth
    digits the sort needs, E evaluated and B blended (pixel, list entry)
    pairs.  Per-unit figures as in the kernel table of the design notes."""
    import torch
    from paper_2410_16978_gb300 import _lib
    lay = _lib.gs_workspace_layout(rast.n, W, H, rast.ws_bytes)
    ws = rast.workspace
    N, V, D = sc.n, int(st.n_visible), int(st.n_dup)
    rec = ws[lay["rec"]:lay["rec"] + 48 * N].view(torch.int32).view(N, 12)
    vis = ws[lay["tiles"]:lay["tiles"] + 4 * N].view(torch.int32) > 0
    rows = ((rec[:, 11] >> 16) & 0xFFFF) - ((rec[:, 10] >> 16) & 0xFFFF)
    R = int(rows[vis].sum().item())
    keys = ws[lay["depth"]:lay["depth"] + 4 * N].view(torch.int32)[vis].to(torch.int64) & 0xFFFFFFFF
    x = int((keys ^ keys.min()).max().item()) | int((keys ^ keys.max()).max().item()) if V else 0
    digits = max(1, (x.bit_length() + 7) // 8)
    ncon = ws[lay["n_contrib"]:lay["n_contrib"] + 4 * W * H].view(torch.int32)
    E = float(ncon.double().sum().item())
    B = float(st.n_blended)
    K = (sc.sh_degree + 1) ** 2
    small = 12 + 12 + 16 + 4 + 1                     # mean, log-scales, quaternion, opacity, layer (FP32)
    Tn = ((W + 15) // 16) * ((H + 15) // 16)
    work = {
        "preprocess": ("hbm", N * (small + 8) + V * (12 * K + 48)),
        "compact": ("hbm", 4 * N + 4 * V),
        "depth_sort": ("hbm", 4 * N + 16 * V + 16 * V * (digits - 1)),
        "bin_rows": ("hbm", 20 * V + 8 * R),
        "bin_tiles": ("hbm", 16 * R + 4 * D + 8 * Tn),
        "composite": ("alu", E * FLOP_EVAL + B * FLOP_BLEND_FWD),
        "composite_bwd": ("alu", E * FLOP_EVAL + B * FLOP_BLEND_BWD),
        "preprocess_bwd": ("hbm", V * (48 + small + 12 * K) + N * (small - 1 + 12 * K)),
        "prune": ("hbm", 9 * N),
    }
    counts = {"gaussians": N, "visible": V, "row_entries": R, "pairs": D, "depth_digits": digits,
              "evaluated_pairs": int(E), "blended_pairs": int(B)}
    return work, counts


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2410_16978_gb300 import (DeviceScene, Rasterizer, _lib, contrib_prune, gs_kernel_launches,
                                        gs_profile_collect, gs_profile_enable)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = build_workload()
    sc, cam = w["scene"], w["cameras"][0]
    W, H = cam.width, cam.height
    bg = tuple(float(v) for v in w["bg"])
    ds = DeviceScene.from_host(sc, device=dev)
    rast = Rasterizer(sc.n, W, H, device=dev)
    image, alpha = rast.render(ds, cam, w["layer_mask"], w["planes"], bg, check=True)   # sizes the pair list
    torch.cuda.synchronize()
    st = rast.status()
    dimg_h, dal_h = _upstream_grads(W, H)
    dimg = torch.from_numpy(dimg_h).to(dev)
    dal = torch.from_numpy(dal_h).to(dev)
    csum = torch.zeros(sc.n, device=dev)
    cmax = torch.zeros(sc.n, device=dev)
    grads = {k: torch.empty(p.shape, dtype=torch.float32, device=dev)
             for k, p in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), ds.params())}
    prune_ws = torch.empty(_lib.gs_prune_workspace_size(sc.n), dtype=torch.uint8, device=dev)
    cam_c = _lib.make_camera(cam)
    cs = ds.c_struct()
    stream = torch.cuda.current_stream(dev)

    def step(dimg_t, dal_t, img_t=image, al_t=alpha):
        csum.zero_()
        cmax.zero_()
        rast.render(ds, cam_c, w["layer_mask"], w["planes"], bg, image=img_t, alpha=al_t, check=False,
                    _c_scene=cs)
        rast.backward(ds, cam_c, bg, dimg_t, dal_t, 0xFFFFFFFF, csum, cmax, grads=grads, _c_scene=cs)
        return contrib_prune(cmax, 0.005, workspace=prune_ws)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step(dimg, dal)
    barrier()

    # ---- the step as one CUDA graph (the same launches, recorded once) ----
    graph, graph_note, step_launches, nk_graph = None, "eager launches", None, None
    if not args.no_graph:
        try:
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):
                step(dimg, dal)
            torch.cuda.current_stream(dev).wait_stream(side)
            torch.cuda.synchronize()
            l_cap = gs_kernel_launches()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                _, _, nk_graph = step(dimg, dal)
            step_launches = gs_kernel_launches() - l_cap
            g.replay()
            torch.cuda.synchronize()
            graph, graph_note = g, "one CUDA graph per step (%d library kernels)" % step_launches
            # a second graph of the same step on a second set of input and output buffers, for the
            # double-buffered end-to-end loop below
            bufs2 = (torch.empty_like(dimg), torch.empty_like(dal), torch.empty_like(image), torch.empty_like(alpha))
            g2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g2):
                _, _, nk_graph2 = step(*bufs2)
            g2.replay()
            torch.cuda.synchronize()
        except Exception as e:          # capture unsupported here: time the eager launches instead
            graph, graph_note = None, "eager launches (graph capture failed: %s)" % str(e).splitlines()[0][:120]
    run_step = graph.replay if graph is not None else (lambda: step(dimg, dal))

    # ---- timed region: device-resident inputs ----
    l0 = gs_kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local_rank) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            evs[k][0].record(stream)
            run_step()
            evs[k][1].record(stream)
        t_end.record(stream)
        barrier()
    launches = (step_launches * args.steps) if graph is not None else (gs_kernel_launches() - l0)
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    per = sorted(a.elapsed_time(b) for a, b in evs)
    ms_step = total_ms / args.steps
    value = whole_job_mpix_s(W * H, args.steps, world, total_ms)

    # ---- stage breakdown: the same steps launched eagerly with the library's event profiler ----
    gs_profile_collect()
    gs_profile_enable(True)
    for _ in range(args.steps):
        step(dimg, dal)
    torch.cuda.synchronize()
    gs_profile_enable(False)
    prof = gs_profile_collect()

    # ---- end to end: host inputs (pinned) and host result every step ----
    # Every step copies its upstream gradients from pinned host memory and reads its image, alpha and kept
    # count back.  With the graphs, the copies run on their own streams into and out of two buffer sets, so
    # step k's upload and step k-1's read-back overlap the compute of steps k-1 and k; each copy waits only
    # for the step that produces or last used its buffers.
    dimg_pin = torch.from_numpy(dimg_h).pin_memory()
    dal_pin = torch.from_numpy(dal_h).pin_memory()
    img_host = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    al_host = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    nk_host = [torch.empty(1, dtype=torch.int64).pin_memory() for _ in range(2)]
    e2e_steps = max(3, min(args.steps, 20))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if graph is not None:
        sets = [(dimg, dal, image, alpha, graph, nk_graph), bufs2[:4] + (g2, nk_graph2)]
        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        up.wait_event(e0)
        down.wait_event(e0)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        for k in range(e2e_steps):
            sb = k % 2
            di, da, im, al, gr, nk = sets[sb]
            with torch.cuda.stream(up):
                if k >= 2:
                    up.wait_event(ev_done[sb])            # step k-2 has consumed this set's inputs
                di.copy_(dimg_pin, non_blocking=True)
                da.copy_(dal_pin, non_blocking=True)
                ev_in[sb].record(up)
            stream.wait_event(ev_in[sb])
            if k >= 2:
                stream.wait_event(ev_out[sb])              # step k-2's results are read back
            gr.replay()
            ev_done[sb].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev_done[sb])
                img_host[sb].copy_(im, non_blocking=True)
                al_host[sb].copy_(al, non_blocking=True)
                nk_host[sb].copy_(nk, non_blocking=True)
                ev_out[sb].record(down)
        for sb in range(2):
            stream.wait_event(ev_out[sb])
        e2e_note = "double-buffered: copies on two copy streams overlap the compute of neighbouring steps"
    else:
        for _ in range(e2e_steps):
            dimg.copy_(dimg_pin, non_blocking=True)
            dal.copy_(dal_pin, non_blocking=True)
            _, _, nk = step(dimg, dal)
            img_host[0].copy_(image, non_blocking=True)
            al_host[0].copy_(alpha, non_blocking=True)
            nk_host[0].copy_(nk, non_blocking=True)
        e2e_note = "serial: copies and compute on one stream"
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_value = world * (W * H) / (e2e_ms / 1e3) / 1e6
    h2d = dimg_h.nbytes + dal_h.nbytes
    d2h = img_host[0].numel() * 4 + al_host[0].numel() * 4 + 8

    # ---- roofline of the dominant kernel ----
    peaks, peaks_src = _peaks()
    stage_ms = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in prof.items()}
    ws_lay = _lib.gs_workspace_layout(rast.n, W, H, rast.ws_bytes)
    ncon = rast.workspace[ws_lay["n_contrib"]:ws_lay["n_contrib"] + 4 * W * H].view(torch.int32)
    pairs_bwd = float(ncon.double().sum().item())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = clk.summary()
    sm_max = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = sms * 128 * 2 * sm_max * 1e6 / 1e12
    dom = max(("composite", "composite_bwd", "preprocess", "preprocess_bwd", "depth_sort", "bin_rows", "bin_tiles"),
              key=lambda k: stage_ms.get(k, 0.0))
    roof_detail = None
    if dom in ("composite", "composite_bwd"):
        blend = FLOP_BLEND_BWD if dom == "composite_bwd" else FLOP_BLEND_FWD
        # per evaluated (pixel, list entry) pair up to n_contrib: the scope table's per-pair figure
        flops = pairs_bwd * (FLOP_S4_PAIR if dom == "composite_bwd" else FLOP_S3_PAIR)
        achieved = flops / (stage_ms[dom] / 1e3) / 1e12
        roof = {"kernel": "k_" + dom, "bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops, "traffic": profiled_traffic(dom),
                "peak_source": "FP32 %d SMs x 128 lanes x 2 x %.0f MHz (sm max)" % (sms, sm_max)}
        # the same with the blend arithmetic only for the pairs actually blended (most evaluated pairs
        # stay below alpha 1/255 and the kernel's block culling never evaluates them)
        blended = float(st.n_blended)
        cons = (pairs_bwd * FLOP_EVAL + blended * blend) / (stage_ms[dom] / 1e3) / 1e12
        roof_detail = {"evaluated_pairs": int(pairs_bwd), "blended_pairs": int(blended),
                       "flop_per_evaluated_pair": FLOP_S4_PAIR if dom == "composite_bwd" else FLOP_S3_PAIR,
                       "achieved_blend_only_tflops": cons, "frac_blend_only": cons / fp32_peak_tflops}
    else:
        K = (sc.sh_degree + 1) ** 2
        per_g = {"preprocess": 12 + 12 + 16 + 4 + 1 + 12 * K + 56, "preprocess_bwd": 2 * (12 + 12 + 16 + 4 + 12 * K) + 48 + 1,
                 "depth_sort": 4 * 24, "bin_rows": 0, "bin_tiles": 0}[dom]
        byts = sc.n * per_g
        achieved = byts / (stage_ms[dom] / 1e3) / 1e9
        roof = {"kernel": "k_" + dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": peaks_src}

    # ---- every step's fraction of its roofline (warm eager stage times) ----
    work, counts = stage_work(rast, sc, st, W, H)
    roof_all = {}
    for k, (bound, amount) in work.items():
        ms = stage_ms.get(k, 0.0)
        if ms <= 0:
            continue
        if bound == "hbm":
            ach = amount / (ms / 1e3) / 1e9
            roof_all[k] = {"ms": round(ms, 4), "bound": "hbm", "bytes": int(amount), "achieved": round(ach, 1),
                           "unit": "GB/s", "peak": peaks["hbm_gbs"], "frac": round(ach / peaks["hbm_gbs"], 4)}
        else:
            ach = amount / (ms / 1e3) / 1e12
            roof_all[k] = {"ms": round(ms, 4), "bound": "alu", "flop": int(amount), "achieved": round(ach, 3),
                           "unit": "TFLOP/s", "peak": round(fp32_peak_tflops, 3),
                           "frac": round(ach / fp32_peak_tflops, 4),
                           "note": "evaluated pairs x %d FLOP + blended pairs x %d" % (
                               FLOP_EVAL, FLOP_BLEND_FWD if k == "composite" else FLOP_BLEND_BWD)}
        tr = profiled_traffic(k)
        if tr is not None:
            roof_all[k]["traffic_bytes"] = tr
            if bound == "hbm":
                roof_all[k]["traffic_over_algorithmic"] = round(tr / amount, 3)
    if "composite_setup" in stage_ms:
        roof_all["composite_setup"] = {"ms": round(stage_ms["composite_setup"], 4), "bound": "latency"}

    # ---- CPU oracle baseline and PSNR check (rank 0, N = 1 only) ----
    cpu, parity, oracle_detail = None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = host_threads()
        v, wall, oracle_detail, parity = oracle_baselines(w, image.cpu().numpy(), threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "one whole step on the full frame (FP64 preprocess of all Gaussians, binning, "
                         "compositing and its backward at every pixel, chain rule, prune) on %d host threads "
                         "over tile rows and Gaussian chunks; %.1f s wall" % (threads, wall)}

    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = run_serving(dev)
    stereo = None
    if rank == 0 and world == 1 and not args.no_stereo:
        stereo = run_stereo(dev)
    training = None
    if rank == 0 and world == 1 and not args.no_training:
        training = run_training(dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_step, "p50_ms": per[len(per) // 2],
                "p99_ms": per[min(len(per) - 1, int(math.ceil(0.99 * len(per))) - 1)],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": _workload_config(w, world),
                "mode": "plain step (one frame per launch sequence): render, backward, prune",
                "launch": graph_note, "counts": counts,
                "psnr_db_vs_fp64_oracle": parity["psnr_db_full_frame"] if parity else None,
                "parity": parity,
                "roofline": roof, "roofline_detail": roof_detail, "roofline_all": roof_all,
                "cpu_baseline": cpu, "oracle_timings": oracle_detail,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": e2e_ms, "copies": e2e_note},
                "clocks": clk, "gpu_launches": int(launches), "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()}}
        if serving:
            tp, ts = serving["trace_plain"], serving["trace_served"]
            line["served"] = {"mpix_s": ts["mpix_s"], "p50_ms": ts["p50_ms"], "p99_ms": ts["p99_ms"],
                              "saturated_mpix_s": serving["saturated_served"]["mpix_s"],
                              "saturated_p99_ms": serving["saturated_served"]["p99_ms"],
                              "psnr_db_vs_fp64_oracle": serving["served_view_psnr_db_vs_fp64_oracle"]}
            line["plain"] = {"mpix_s": tp["mpix_s"], "p50_ms": tp["p50_ms"], "p99_ms": tp["p99_ms"],
                             "saturated_mpix_s": serving["saturated_plain"]["mpix_s"],
                             "saturated_p99_ms": serving["saturated_plain"]["p99_ms"]}
        line.update(serving=serving, stereo=stereo, training=training)
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-training", action="store_true")
    ap.add_argument("--no-stereo", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of one CUDA graph per step")
    args = ap.parse_args()
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Serving loop: several layered models resident on the device, render
requests of mixed resolution, layer mask and clip planes admitted by a device
memory budget and composited in batches (continuous batching), next to the
plain path that renders one request per launch sequence.

The paper's renderer keeps a layered model in GPU buffers and re-renders it
every frame with layers toggled or cut, once per eye (Sec. 3.3); this module
serves many such views at once.  Every view still goes through the CUDA path
of libgs.so: ``gs_render_batch`` runs each view's preprocess and sorts and
then composites all views of a batch with one persistent launch.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib
from .api import DeviceScene

SCENE_MARGIN = 1.25     # pair capacity = calibrated pairs of a (model, size) x this margin


@dataclasses.dataclass
class RenderRequest:
    rid: int
    model: str
    cameras: list                  # 1 camera, or 2 for a stereo pair
    layer_mask: int = 0xFFFFFFFF
    planes: tuple = ()
    bg: tuple = (0.0, 0.0, 0.0)
    arrival: float = 0.0           # seconds from the start of the trace

    @property
    def pixels(self) -> int:
        return sum(int(c.width) * int(c.height) for c in self.cameras)


@dataclasses.dataclass
class RequestResult:
    rid: int
    arrival: float
    start: float = math.nan        # host time the request was launched
    done: float = math.nan         # device completion time
    images: Optional[list] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _ViewBuffers:
    """Workspace, outputs and a pinned status word of one in-flight view."""

    def __init__(self, n: int, W: int, H: int, cap: int, device):
        self.cap = int(cap)
        self.ws_bytes = _lib.gs_render_workspace_size(n, W, H, cap)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.image = torch.empty((3, H, W), dtype=torch.float32, device=device)
        self.alpha = torch.empty((H, W), dtype=torch.float32, device=device)
        ctl = _lib.gs_workspace_layout(n, W, H, self.ws_bytes)["ctl"]
        self.status_dev = self.workspace[ctl:ctl + ctypes.sizeof(_lib.gs_status)]
        self.status_host = torch.empty(ctypes.sizeof(_lib.gs_status), dtype=torch.uint8, pin_memory=True)
        self.bytes = self.ws_bytes + self.image.numel() * 4 + self.alpha.numel() * 4

    def fetch_status(self):
        """Enqueues the copy of the status word on the current stream."""
        self.status_host.copy_(self.status_dev, non_blocking=True)

    def status(self) -> _lib.gs_status:
        return _lib.gs_status.from_buffer_copy(self.status_host.numpy().tobytes())


class RenderServer:
    """Renders requests against resident models.

    ``memory_budget`` caps the bytes of view buffers in flight; a request is
    admitted when all of its views fit next to those already in flight (a
    request larger than the whole budget runs alone).  Buffers are pooled per
    (model, width, height) and reused, so the steady state allocates nothing.
    A view whose (tile, Gaussian) pairs overflowed its workspace is detected
    from its status word when its batch retires; the capacity of that (model,
    size) grows and the request is rendered again."""

    def __init__(self, models: Dict[str, DeviceScene], memory_budget: int = 8 << 30, max_views_per_batch: int = 16,
                 max_inflight_batches: int = 2, device="cuda", policy: str = "priority",
                 large_view_pixels: int = 2_000_000):
        if policy not in ("priority", "fifo"):
            raise ValueError(policy)
        self.models = models
        self.device = torch.device(device)
        self.budget = int(memory_budget)
        self.max_views = min(int(max_views_per_batch), _lib.GS_MAX_BATCH)
        self.max_inflight = int(max_inflight_batches)
        self.policy = policy
        self.large_view_pixels = int(large_view_pixels)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.max_inflight)]
        self.stream_hi = torch.cuda.Stream(self.device, priority=-1)
        self._cap: Dict[tuple, int] = {}
        self._free: Dict[tuple, List[_ViewBuffers]] = collections.defaultdict(list)
        self._c_scene = {k: m.c_struct() for k, m in models.items()}
        self.in_use = 0
        self.retries = 0
        self.batches = 0
        self.views_launched = 0

    # -- sizing ---------------------------------------------------------------
    def calibrate(self, model: str, cameras, layer_mask=0xFFFFFFFF, planes=()) -> int:
        """Renders the given views with status checks and sizes the pair
        capacity of (model, size) at SCENE_MARGIN x the largest count seen."""
        from .api import Rasterizer
        m = self.models[model]
        for cam in cameras:
            r = Rasterizer(m.n, cam.width, cam.height, device=self.device)
            r.render(m, cam, layer_mask, planes, check=True)
            need = int(r.status().n_dup)
            key = self._key(model, cam)
            self._cap[key] = max(self._cap.get(key, 0), int(need * SCENE_MARGIN) + 4096)
        return max(v for k, v in self._cap.items() if k[0] == model)

    def _key(self, model, cam):
        return (model, int(cam.width), int(cam.height))

    def _cap_of(self, key) -> int:
        return self._cap.get(key, max(1 << 16, 8 * self.models[key[0]].n))

    def view_bytes(self, model: str, cam) -> int:
        key = self._key(model, cam)
        return (_lib.gs_render_workspace_size(self.models[model].n, cam.width, cam.height, self._cap_of(key))
                + 16 * int(cam.width) * int(cam.height))

    def request_bytes(self, req: RenderRequest) -> int:
        return sum(self.view_bytes(req.model, c) for c in req.cameras)

    def _take(self, model, cam) -> _ViewBuffers:
        key = self._key(model, cam)
        vb = self._free[key].pop() if self._free[key] else \
            _ViewBuffers(self.models[model].n, cam.width, cam.height, self._cap_of(key), self.device)
        self.in_use += vb.bytes
        return vb

    def _give(self, model, cam, vb: _ViewBuffers):
        self.in_use -= vb.bytes
        key = self._key(model, cam)
        if vb.cap >= self._cap_of(key):
            self._free[key].append(vb)

    def release_pool(self):
        self._free.clear()

    # -- launches -------------------------------------------------------------
    def _launch_plain(self, req: RenderRequest, stream: torch.cuda.Stream, keep_images: bool):
        """The plain path: one gs_render call per view of one request."""
        views = []
        cs = self._c_scene[req.model]
        with torch.cuda.stream(stream):
            for cam in req.cameras:
                vb = self._take(req.model, cam)
                _lib.gs_render(cs, _lib.make_camera(cam), req.layer_mask, list(req.planes), req.bg, vb.workspace,
                               vb.ws_bytes, vb.image, vb.alpha, int(stream.cuda_stream))
                vb.fetch_status()
                views.append((req, cam, vb))
            imgs = {req.rid: [vb.image.clone() for _, _, vb in views]} if keep_images else None
        self.views_launched += len(views)
        return views, imgs

    def _launch_batch(self, reqs: Sequence[RenderRequest], stream: torch.cuda.Stream, keep_images: bool):
        """All views of ``reqs`` in one gs_render_batch call."""
        items, views = [], []
        for req in reqs:
            cs = self._c_scene[req.model]
            for cam in req.cameras:
                vb = self._take(req.model, cam)
                views.append((req, cam, vb))
                items.append(dict(scene=cs, camera=_lib.make_camera(cam), layer_mask=req.layer_mask,
                                  planes=list(req.planes), bg=req.bg, workspace=vb.workspace, ws_bytes=vb.ws_bytes,
                                  image=vb.image, alpha=vb.alpha))
        _lib.gs_render_batch(items, int(stream.cuda_stream))
        imgs = None
        with torch.cuda.stream(stream):
            for _, _, vb in views:
                vb.fetch_status()
            if keep_images:
                imgs = {}
                for req, cam, vb in views:
                    imgs.setdefault(req.rid, []).append(vb.image.clone())
        self.batches += 1
        self.views_launched += len(views)
        return views, imgs

    # -- trace replay ---------------------------------------------------------
    def is_large(self, req: RenderRequest) -> bool:
        return any(int(c.width) * int(c.height) >= self.large_view_pixels for c in req.cameras)

    def run_trace(self, requests: Sequence[RenderRequest], mode: str = "served", keep_images=False):
        """Replays the arrival trace in real time.  Returns (results, seconds
        from the first arrival to the last completion).  Completion times are
        device event times, on the clock of the trace.

        plain:  one request at a time in arrival order, one gs_render call per
                view, all on one stream (up to max_inflight requests queued).
        served: continuous batching.  Waiting requests are packed, in arrival
                order, into gs_render_batch launches of up to max_views views
                as soon as a launch slot and the memory budget allow.  With
                policy "priority" there are two lanes: requests with a view of
                at least large_view_pixels go to a high-priority stream, one
                batch at a time; the others to normal-priority streams, so
                small requests fill the device around a large frame without
                delaying it.  Policy "fifo" is one lane over all streams."""
        if mode not in ("served", "plain"):
            raise ValueError(mode)
        reqs = sorted(requests, key=lambda r: r.arrival)
        results = {r.rid: RequestResult(r.rid, r.arrival) for r in reqs}
        torch.cuda.synchronize(self.device)
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(self.streams[0])
        ref.synchronize()
        t0 = time.perf_counter()
        if mode == "plain":
            lanes = [dict(pred=lambda r: True, streams=[self.streams[0]], slots=self.max_inflight, batch=False)]
        elif self.policy == "fifo":
            lanes = [dict(pred=lambda r: True, streams=self.streams, slots=self.max_inflight, batch=True)]
        else:
            lanes = [dict(pred=self.is_large, streams=[self.stream_hi], slots=1, batch=True),
                     dict(pred=lambda r: not self.is_large(r), streams=self.streams, slots=self.max_inflight,
                          batch=True)]
        for ln in lanes:
            ln.update(waiting=collections.deque(), pending=[], k=0)
        nxt = 0

        def lane_of(r):
            return next(ln for ln in lanes if ln["pred"](r))

        while nxt < len(reqs) or any(ln["waiting"] or ln["pending"] for ln in lanes):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                lane_of(reqs[nxt])["waiting"].append(reqs[nxt])
                nxt += 1
            for ln in lanes:
                redo = collections.deque()
                self._retire(ln["pending"], results, ref, redo)
                ln["waiting"].extendleft(reversed(redo))
            launched = False
            for ln in lanes:
                waiting, pending = ln["waiting"], ln["pending"]
                if not waiting or len(pending) >= ln["slots"]:
                    continue
                batch, nviews, nbytes = [], 0, 0
                busy = any(l2["pending"] for l2 in lanes)
                while waiting:
                    r = waiting[0]
                    if not ln["batch"] and batch:
                        break
                    if nviews + len(r.cameras) > self.max_views:
                        break
                    rb = self.request_bytes(r)
                    if self.in_use + nbytes + rb > self.budget and (batch or busy):
                        break
                    batch.append(waiting.popleft())
                    nviews += len(r.cameras)
                    nbytes += rb
                if not batch:
                    continue
                stream = ln["streams"][ln["k"] % len(ln["streams"])]
                ln["k"] += 1
                st = time.perf_counter() - t0
                for r in batch:
                    if math.isnan(results[r.rid].start):
                        results[r.rid].start = st
                if ln["batch"]:
                    views, imgs = self._launch_batch(batch, stream, keep_images)
                else:
                    views, imgs = self._launch_plain(batch[0], stream, keep_images)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                pending.append((ev, views, imgs))
                launched = True
            if launched:
                continue
            if not any(ln["pending"] or ln["waiting"] for ln in lanes) and nxt < len(reqs):
                wait = reqs[nxt].arrival - (time.perf_counter() - t0)
                if wait > 3e-4:
                    time.sleep(wait - 2e-4)
        last = max(r.done for r in results.values())
        return [results[r.rid] for r in reqs], last - reqs[0].arrival

    def _retire(self, pending, results, ref, waiting):
        keep = []
        for ev, views, imgs in pending:
            if not ev.query():
                keep.append((ev, views, imgs))
                continue
            t = ref.elapsed_time(ev) / 1e3
            redo = {}
            for req, cam, vb in views:
                stt = vb.status()
                if stt.error == _lib.GS_ERR_WORKSPACE:
                    key = self._key(req.model, cam)
                    self._cap[key] = max(self._cap_of(key), int(stt.n_dup * SCENE_MARGIN) + 4096)
                    redo[req.rid] = req
                elif stt.error != _lib.GS_OK:
                    raise _lib.GsError(stt.error, "device status of request %d" % req.rid)
            for req, cam, vb in views:
                if req.rid not in redo:
                    results[req.rid].done = t
                    if imgs:
                        results[req.rid].images = imgs.get(req.rid)
                self._give(req.model, cam, vb)
            for req in reversed(list(redo.values())):
                self.retries += 1
                waiting.appendleft(req)
        pending[:] = keep


def summarize(results: Sequence[RequestResult], requests: Sequence[RenderRequest], wall: float) -> dict:
    """Throughput over the replay and latency percentiles, overall and per
    request size ("WxHxeyes")."""
    lat = np.array([r.latency for r in results]) * 1e3
    px = sum(r.pixels for r in requests)
    size_of = {q.rid: "%dx%dx%d" % (q.cameras[0].width, q.cameras[0].height, len(q.cameras)) for q in requests}
    by = collections.defaultdict(list)
    for r in results:
        by[size_of[r.rid]].append(r.latency * 1e3)
    return {"mpix_s": px / wall / 1e6, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "requests": len(results), "wall_s": wall, "mpixels": px / 1e6,
            "by_size_p50_p99_ms": {k: [round(float(np.percentile(v, 50)), 4), round(float(np.percentile(v, 99)), 4)]
                                   for k, v in sorted(by.items())}}


def make_trace(rng: np.random.Generator, model_names: Sequence[str], n_requests=512, rate=300.0,
               sizes=((512, 512, 1), (1024, 1024, 1), (2064, 2208, 2)), n_planes_max=2, radius=4.0):
    """Poisson arrivals at ``rate`` per second (all at time 0 when ``rate`` is
    None); each request picks a model, a size (the last with two eyes 64 mm
    apart), a random 5-bit layer mask, 0..n random clip planes, a random
    viewpoint on a sphere and a random background."""
    import synth
    t = 0.0
    out = []
    for rid in range(n_requests):
        if rate is not None:
            t += rng.exponential(1.0 / rate)
        model = model_names[int(rng.integers(len(model_names)))]
        W, H, eyes = sizes[int(rng.integers(len(sizes)))]
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        cam = synth.look_at_camera(radius * d, fov_x_deg=50.0, width=W, height=H)
        cams = list(synth.stereo_pair(cam, 0.064)) if eyes == 2 else [cam]
        planes = synth.random_clip_planes(rng, int(rng.integers(0, n_planes_max + 1)))
        out.append(RenderRequest(rid, model, cams, int(rng.integers(1, 32)), tuple(planes),
                                 tuple(float(v) for v in rng.uniform(0, 1, 3)), t))
    return out

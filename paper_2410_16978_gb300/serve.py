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
import threading
import time
from typing import Callable, Dict, List, Optional, Sequence

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
    cancel_at: Optional[float] = None   # trace time at which the client withdraws it (if not yet launched)

    @property
    def pixels(self) -> int:
        return sum(int(c.width) * int(c.height) for c in self.cameras)


@dataclasses.dataclass
class RequestResult:
    rid: int
    arrival: float
    start: float = math.nan        # host time the request was launched
    done: float = math.nan         # device completion time (or the time it was cancelled / failed)
    images: Optional[list] = None
    status: str = "pending"        # "done", "cancelled" (withdrawn before launch) or "failed"
    error: int = 0                 # GS_ERR_* of a failed request (GS_ERR_OOM: no device memory for its views)

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
    size) grows and the request is rendered again.

    Failures and withdrawals.  When the device cannot hold a request's view
    buffers (the allocation raises), the server drops its buffer pools and
    tries once more; if that fails too, that request alone ends with status
    "failed" and error GS_ERR_OOM and the others go on.  ``cancel(rid)`` (any
    thread) or a request's ``cancel_at`` withdraws a request that has not been
    launched yet; it ends with status "cancelled" and nothing of it runs on
    the device.  ``allocate(n, W, H, capacity, device)`` makes a view's
    buffers (``_ViewBuffers`` by default; tests inject failures there)."""

    def __init__(self, models: Dict[str, DeviceScene], memory_budget: int = 8 << 30, max_views_per_batch: int = 16,
                 max_inflight_batches: int = 2, device="cuda", policy: str = "priority",
                 large_view_pixels: int = 2_000_000, allocate: Optional[Callable] = None, large_slots: int = 2,
                 split_large: bool = True, split_small: bool = True):
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
        self.large_slots = max(1, int(large_slots))
        self.split_large = bool(split_large)
        self.split_small = bool(split_small)
        self.streams_hi = [torch.cuda.Stream(self.device, priority=-1) for _ in range(self.large_slots)]
        self.stream_hi = self.streams_hi[0]
        # a companion stream per stream: the views of a batch are split between the two, so the two eyes of
        # a stereo request (or two halves of a batch of small views) render side by side
        self.split_hi = {hs.cuda_stream: torch.cuda.Stream(self.device, priority=-1) for hs in self.streams_hi}
        self.split_hi.update({ns.cuda_stream: torch.cuda.Stream(self.device) for ns in self.streams})
        self._cap: Dict[tuple, int] = {}
        self._free: Dict[tuple, List[_ViewBuffers]] = collections.defaultdict(list)
        self._c_scene = {k: m.c_struct() for k, m in models.items()}
        self._allocate = allocate if allocate is not None else _ViewBuffers
        self._cancel_lock = threading.Lock()
        self._cancelled = set()
        self.in_use = 0
        self.retries = 0
        self.batches = 0
        self.views_launched = 0
        self.failed = 0
        self.cancelled = 0

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

    def capacities(self) -> Dict[tuple, int]:
        """The pair capacity per (model, width, height), e.g. to restore a
        calibration later with ``set_capacities``."""
        return dict(self._cap)

    def set_capacities(self, caps: Dict[tuple, int]):
        """Replaces the pair capacities and drops the pooled buffers."""
        self._cap = dict(caps)
        self.release_pool()

    def cancel(self, rid: int):
        """Withdraws request ``rid`` if it has not been launched yet (callable
        from any thread; a launched request completes normally)."""
        with self._cancel_lock:
            self._cancelled.add(int(rid))

    def _take(self, model, cam) -> _ViewBuffers:
        key = self._key(model, cam)
        cap = self._cap_of(key)
        pool = self._free[key]
        while pool and pool[-1].cap < cap:        # sized before the capacity last grew
            pool.pop()
        if pool:
            vb = pool.pop()
        else:
            try:
                vb = self._allocate(self.models[model].n, cam.width, cam.height, cap, self.device)
            except torch.cuda.OutOfMemoryError as e:
                raise _lib.GsError(_lib.GS_ERR_OOM, "view buffers of %s %dx%d: %s" % (
                    model, cam.width, cam.height, str(e).splitlines()[0] if str(e) else "out of memory")) from e
        self.in_use += vb.bytes
        return vb

    def _give(self, model, cam, vb: _ViewBuffers):
        self.in_use -= vb.bytes
        key = self._key(model, cam)
        if vb.cap >= self._cap_of(key):
            self._free[key].append(vb)

    def _acquire(self, req: RenderRequest):
        """The view buffers of every view of ``req``; on GS_ERR_OOM the pools
        are dropped and the allocation is tried once more.  Raises GsError
        (GS_ERR_OOM) when that fails too, holding nothing."""
        for attempt in range(2):
            got = []
            try:
                for cam in req.cameras:
                    got.append((req, cam, self._take(req.model, cam)))
                return got
            except _lib.GsError as e:
                for r, cam, vb in got:
                    self._give(r.model, cam, vb)
                if e.code != _lib.GS_ERR_OOM or attempt == 1:
                    raise
                self.release_pool()
                torch.cuda.empty_cache()

    def release_pool(self):
        self._free.clear()

    # -- launches -------------------------------------------------------------
    def _launch_plain(self, views, stream: torch.cuda.Stream, keep_images: bool):
        """The plain path: one gs_render call per view of one request
        (``views``: its (request, camera, buffers) triples)."""
        with torch.cuda.stream(stream):
            for req, cam, vb in views:
                _lib.gs_render(self._c_scene[req.model], _lib.make_camera(cam), req.layer_mask, list(req.planes),
                               req.bg, vb.workspace, vb.ws_bytes, vb.image, vb.alpha, int(stream.cuda_stream))
                vb.fetch_status()
            imgs = {views[0][0].rid: [vb.image.clone() for _, _, vb in views]} if keep_images else None
        self.views_launched += len(views)
        return views, imgs

    def _launch_batch(self, views, stream: torch.cuda.Stream, keep_images: bool, split: bool = False):
        """All ``views`` ((request, camera, buffers) triples of several
        requests) in one gs_render_batch call on ``stream``; with ``split``
        (and two views or more) the second half of the views goes to the
        stream's companion stream in a second call, and ``stream`` waits for
        it, so both halves render side by side and one event on ``stream``
        still marks the end of the batch."""
        def items_of(vs):
            return [dict(scene=self._c_scene[req.model], camera=_lib.make_camera(cam), layer_mask=req.layer_mask,
                         planes=list(req.planes), bg=req.bg, workspace=vb.workspace, ws_bytes=vb.ws_bytes,
                         image=vb.image, alpha=vb.alpha) for req, cam, vb in vs]
        aux = self.split_hi.get(stream.cuda_stream) if split and len(views) >= 2 else None
        if aux is not None:
            half = (len(views) + 1) // 2
            aux.wait_stream(stream)                     # the companion starts after what the lane queued before
            _lib.gs_render_batch(items_of(views[:half]), int(stream.cuda_stream))
            _lib.gs_render_batch(items_of(views[half:]), int(aux.cuda_stream))
            with torch.cuda.stream(aux):
                for _, _, vb in views[half:]:
                    vb.fetch_status()
            stream.wait_stream(aux)
        else:
            _lib.gs_render_batch(items_of(views), int(stream.cuda_stream))
        imgs = None
        with torch.cuda.stream(stream):
            for _, _, vb in (views if aux is None else views[:half]):
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
                at least large_view_pixels go to large_slots high-priority
                streams, one batch in flight on each (two let one large frame's
                preprocess and sorts overlap another's compositing); the others
                to normal-priority streams, so small requests fill the device
                around the large frames without delaying them.  Policy "fifo"
                is one lane over all streams."""
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
            lanes = [dict(pred=self.is_large, streams=self.streams_hi, slots=self.large_slots, batch=True,
                          split=self.split_large),
                     dict(pred=lambda r: not self.is_large(r), streams=self.streams, slots=self.max_inflight,
                          batch=True, split=self.split_small)]
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
            self._withdraw(lanes, results, now)
            launched = False
            for ln in lanes:
                waiting, pending = ln["waiting"], ln["pending"]
                if not waiting or len(pending) >= ln["slots"]:
                    continue
                batch, views, nviews, nbytes = [], [], 0, 0
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
                    waiting.popleft()
                    try:
                        got = self._acquire(r)
                    except _lib.GsError as e:
                        res = results[r.rid]
                        res.status, res.error, res.done = "failed", e.code, time.perf_counter() - t0
                        self.failed += 1
                        continue
                    batch.append(r)
                    views += got
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
                    views, imgs = self._launch_batch(views, stream, keep_images, ln.get("split", False))
                else:
                    views, imgs = self._launch_plain(views, stream, keep_images)
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
        ends = [r.done for r in results.values() if r.status == "done"]
        last = max(ends) if ends else reqs[0].arrival
        return [results[r.rid] for r in reqs], last - reqs[0].arrival

    def _withdraw(self, lanes, results, now):
        """Drops waiting (not yet launched) requests that were cancelled."""
        with self._cancel_lock:
            ids = set(self._cancelled)
        for ln in lanes:
            keep = collections.deque()
            for r in ln["waiting"]:
                if r.rid in ids or (r.cancel_at is not None and r.cancel_at <= now):
                    res = results[r.rid]
                    if res.status == "pending":
                        res.status, res.done = "cancelled", now
                        self.cancelled += 1
                    continue
                keep.append(r)
            ln["waiting"] = keep

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
                    self._free[key].clear()          # pooled buffers of the old capacity would overflow again
                    redo[req.rid] = req
                elif stt.error != _lib.GS_OK:
                    raise _lib.GsError(stt.error, "device status of request %d" % req.rid)
            for req, cam, vb in views:
                if req.rid not in redo:
                    results[req.rid].done = t
                    results[req.rid].status = "done"
                    if imgs:
                        results[req.rid].images = imgs.get(req.rid)
                self._give(req.model, cam, vb)
            for req in reversed(list(redo.values())):
                self.retries += 1
                waiting.appendleft(req)
        pending[:] = keep


def summarize(results: Sequence[RequestResult], requests: Sequence[RenderRequest], wall: float) -> dict:
    """Throughput over the replay and latency percentiles of the completed
    requests, overall and per request size ("WxHxeyes"), with the counts of
    cancelled and failed ones."""
    done = [r for r in results if r.status == "done" or (r.status == "pending" and np.isfinite(r.done))]
    lat = np.array([r.latency for r in done]) * 1e3
    done_ids = {r.rid for r in done}
    px = sum(q.pixels for q in requests if q.rid in done_ids)
    size_of = {q.rid: "%dx%dx%d" % (q.cameras[0].width, q.cameras[0].height, len(q.cameras)) for q in requests}
    by = collections.defaultdict(list)
    for r in done:
        by[size_of[r.rid]].append(r.latency * 1e3)
    pct = (lambda a, q: float(np.percentile(a, q))) if lat.size else (lambda a, q: math.nan)
    return {"mpix_s": px / wall / 1e6 if wall > 0 else 0.0, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "mean_ms": float(lat.mean()) if lat.size else math.nan, "requests": len(done), "wall_s": wall,
            "mpixels": px / 1e6, "cancelled": sum(r.status == "cancelled" for r in results),
            "failed": sum(r.status == "failed" for r in results),
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

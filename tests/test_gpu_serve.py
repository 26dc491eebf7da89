"""Serving loop on the GPU: every request's images are the same when served in
a mixed continuous batch as when the request is rendered alone, including a
request re-rendered after its pair list overflowed; plain and served replays
of one trace give the same images."""
import numpy as np
import pytest
import torch

import synth
from paper_2410_16978_gb300 import DeviceScene, Rasterizer
from paper_2410_16978_gb300.serve import RenderServer, make_trace, summarize

pytestmark = pytest.mark.gpu

SIZES = ((64, 64, 1), (128, 96, 1), (80, 72, 2))


def _models():
    rng = np.random.default_rng(11)
    out = {}
    for name, scale in (("m_small", 0.004), ("m_mid", 0.01), ("m_big", 0.02)):
        counts = [max(1, int(c * scale)) for c in synth.scenes.C2_COUNTS]
        out[name] = DeviceScene.from_host(synth.shell_scene(rng, counts, synth.scenes.C2_RADII))
    return out


def _alone(ds, req):
    imgs = []
    for cam in req.cameras:
        r = Rasterizer(ds.n, cam.width, cam.height)
        img, _ = r.render(ds, cam, req.layer_mask, req.planes, req.bg, check=True)
        imgs.append(img)
    torch.cuda.synchronize()
    return imgs


def test_served_mix_equals_alone():
    models = _models()
    trace = make_trace(np.random.default_rng(3), list(models), n_requests=48, rate=4000.0, sizes=SIZES)
    # 128x96 and the stereo 80x72 views count as large: both lanes are used
    srv = RenderServer(models, memory_budget=64 << 20, max_views_per_batch=8, large_view_pixels=5000)
    # a capacity far below the need of one model forces the overflow-and-retry path
    srv._cap[("m_big", 128, 96)] = 64
    res, wall = srv.run_trace(trace, "served", keep_images=True)
    torch.cuda.synchronize()
    assert srv.retries >= 1
    assert srv.batches < len(trace)          # requests were batched together
    assert srv.in_use == 0
    by = {r.rid: r for r in res}
    for req in trace:
        got = by[req.rid].images
        assert got is not None and len(got) == len(req.cameras)
        for a, b in zip(got, _alone(models[req.model], req)):
            assert torch.equal(a, b), req.rid
    s = summarize(res, trace, wall)
    assert s["requests"] == len(trace) and s["p99_ms"] >= s["p50_ms"] > 0
    assert all(r.done >= r.arrival for r in res)


def test_plain_and_served_replays_agree():
    models = _models()
    trace = make_trace(np.random.default_rng(4), list(models), n_requests=24, rate=2000.0, sizes=SIZES)
    srv = RenderServer(models, memory_budget=32 << 20, policy="fifo")
    a, _ = srv.run_trace(trace, "plain", keep_images=True)
    b, _ = srv.run_trace(trace, "served", keep_images=True)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert x.rid == y.rid
        for p, q in zip(x.images, y.images):
            assert torch.equal(p, q), x.rid


def test_budget_bounds_memory_in_flight():
    """With a budget below one request, requests still complete one at a time."""
    models = _models()
    trace = make_trace(np.random.default_rng(5), list(models), n_requests=10, rate=None, sizes=SIZES)
    srv = RenderServer(models, memory_budget=1)
    res, _ = srv.run_trace(trace, "served")
    assert srv.batches == len(trace) + srv.retries
    assert all(np.isfinite(r.done) for r in res)


def test_out_of_memory_fails_only_that_request():
    """An allocation failure of one request's view buffers (injected in the
    allocator, as the device would raise it) ends that request with
    GS_ERR_OOM after one retry with the pools dropped; every other request
    completes with the same images as alone."""
    from paper_2410_16978_gb300 import _lib
    from paper_2410_16978_gb300.serve import _ViewBuffers
    models = _models()
    trace = make_trace(np.random.default_rng(6), list(models), n_requests=16, rate=None, sizes=SIZES)
    victim = next(r for r in trace if r.model == "m_mid")
    calls = {"n": 0, "refused": 0}
    in_victim = {"on": False}

    def allocate(n, W, H, cap, device):
        calls["n"] += 1
        if in_victim["on"]:
            calls["refused"] += 1
            raise torch.cuda.OutOfMemoryError("CUDA out of memory (injected)")
        return _ViewBuffers(n, W, H, cap, device)

    srv = RenderServer(models, memory_budget=64 << 20, allocate=allocate)
    real_acquire = srv._acquire

    def acquire(req):
        in_victim["on"] = req.rid == victim.rid
        try:
            return real_acquire(req)
        finally:
            in_victim["on"] = False

    srv._acquire = acquire
    res, wall = srv.run_trace(trace, "served", keep_images=True)
    torch.cuda.synchronize()
    by = {r.rid: r for r in res}
    assert by[victim.rid].status == "failed" and by[victim.rid].error == _lib.GS_ERR_OOM
    assert by[victim.rid].images is None
    assert calls["refused"] == 2                  # the first attempt and the retry after the pools were dropped
    assert srv.failed == 1 and srv.in_use == 0
    for req in trace:
        if req.rid == victim.rid:
            continue
        assert by[req.rid].status == "done"
        for a, b in zip(by[req.rid].images, _alone(models[req.model], req)):
            assert torch.equal(a, b), req.rid
    s = summarize(res, trace, wall)
    assert s["failed"] == 1 and s["requests"] == len(trace) - 1


def test_cancelled_requests_never_launch():
    """Requests withdrawn before launch (by cancel_at on the trace clock, and
    by cancel() from another thread before the replay starts) end as
    "cancelled", launch no view, and leave the other results unchanged."""
    import dataclasses
    import threading
    models = _models()
    base = make_trace(np.random.default_rng(7), list(models), n_requests=20, rate=None, sizes=SIZES)
    # everything arrives at 0; two requests arrive late and are withdrawn before they arrive
    trace = [dataclasses.replace(r, arrival=0.05, cancel_at=0.0) if k in (3, 11) else r for k, r in enumerate(base)]
    srv = RenderServer(models, memory_budget=64 << 20)
    t = threading.Thread(target=srv.cancel, args=(trace[7].rid,))
    t.start()
    t.join()
    res, wall = srv.run_trace(trace, "served", keep_images=True)
    torch.cuda.synchronize()
    by = {r.rid: r for r in res}
    gone = {trace[3].rid, trace[11].rid, trace[7].rid}
    for rid in gone:
        assert by[rid].status == "cancelled" and by[rid].images is None
    assert srv.cancelled == 3 and srv.retries == 0
    assert srv.views_launched == sum(len(r.cameras) for r in trace if r.rid not in gone)
    for req in trace:
        if req.rid in gone:
            continue
        assert by[req.rid].status == "done"
        for a, b in zip(by[req.rid].images, _alone(models[req.model], req)):
            assert torch.equal(a, b), req.rid
    s = summarize(res, trace, wall)
    assert s["cancelled"] == 3 and s["requests"] == len(trace) - 3


def test_capacity_growth_drops_undersized_pooled_buffers():
    """After an overflow grows a (model, size) capacity, no pooled buffer of
    the old capacity is handed out again."""
    models = _models()
    cam = synth.look_at_camera((0.3, -0.2, 3.6), width=128, height=96)
    srv = RenderServer(models, memory_budget=64 << 20)
    key = ("m_big", 128, 96)
    srv._cap[key] = 64
    vbs = [srv._take("m_big", cam) for _ in range(3)]
    for vb in vbs:
        srv._give("m_big", cam, vb)
    assert len(srv._free[key]) == 3
    srv._cap[key] = 1 << 20                      # the capacity grew after these were pooled
    vb = srv._take("m_big", cam)
    assert vb.cap == 1 << 20 and len(srv._free[key]) == 0
    srv._give("m_big", cam, vb)

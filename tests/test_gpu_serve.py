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

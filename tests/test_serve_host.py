"""Host logic of the serving loop (no GPU): the request trace and the latency
summary."""
import numpy as np

import synth
from paper_2410_16978_gb300.serve import RenderRequest, RequestResult, make_trace, summarize


def test_trace_shape():
    sizes = ((512, 512, 1), (1024, 1024, 1), (2064, 2208, 2))
    tr = make_trace(np.random.default_rng(0), ["a", "b", "c"], n_requests=400, rate=300.0, sizes=sizes)
    arr = np.array([r.arrival for r in tr])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 300) < 0.25 / 300          # exponential gaps, mean 1/rate
    assert abs(np.median(gaps) - np.log(2) / 300) < 0.3 / 300
    assert {r.model for r in tr} == {"a", "b", "c"}
    for r in tr:
        assert 1 <= r.layer_mask <= 31 and len(r.planes) <= 2
        dims = {(c.width, c.height) for c in r.cameras}
        assert len(dims) == 1
        w, h = dims.pop()
        assert (w, h, len(r.cameras)) in sizes
        if len(r.cameras) == 2:
            l, rr = r.cameras
            cl = -l.R.T @ l.t
            cr = -rr.R.T @ rr.t
            assert abs(np.linalg.norm(cl - cr) - 0.064) < 1e-5
    assert make_trace(np.random.default_rng(0), ["a"], 5, rate=None)[-1].arrival == 0.0


def test_summary_percentiles():
    cam = synth.look_at_camera((0, 0, 4), width=100, height=50)
    reqs = [RenderRequest(k, "a", [cam], arrival=0.01 * k) for k in range(100)]
    res = [RequestResult(k, 0.01 * k, done=0.01 * k + 0.001 * (k + 1)) for k in range(100)]
    s = summarize(res, reqs, 2.0)
    assert abs(s["p50_ms"] - 50.5) < 1e-9 and abs(s["p99_ms"] - 99.01) < 1e-9
    assert abs(s["mpix_s"] - 100 * 5000 / 2.0 / 1e6) < 1e-12

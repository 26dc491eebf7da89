"""Pins of the oracle's single-precision decision path against its FP64
definition: the same projection, with integer decisions (culls, radius, tile
rectangle, depth key) taken in IEEE single precision in a fixed order."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_expf32_error_bound():
    xs = np.concatenate([np.linspace(-80, 80, 20001), np.linspace(-1, 1, 2001),
                         np.random.default_rng(0).uniform(-20, 20, 5000)]).astype(np.float32)
    got = oracle.expf32(xs).astype(np.float64)
    want = np.exp(xs.astype(np.float64))
    rel = np.abs(got - want) / want
    assert rel.max() < 2.0 ** -21          # within 4 units in the last place
    assert oracle.expf32([0.0])[0] == 1.0


def test_expf32_saturates_outside_range():
    assert oracle.expf32([200.0])[0] == oracle.expf32([80.0])[0]
    assert oracle.expf32([-200.0])[0] == oracle.expf32([-80.0])[0] > 0


def _compare(sc, cam, mask=0xFFFFFFFF, planes=()):
    p64 = oracle.preprocess(sc, cam, mask, planes, "f64")
    p32 = oracle.preprocess(sc, cam, mask, planes, "f32")
    return p64, p32


@pytest.mark.parametrize("which", ["c1", "c2_small"])
def test_f32_path_tracks_f64_definition(which):
    if which == "c1":
        w = synth.scene_c1()
    else:
        w = synth.scene_c2(scale=0.01, width=256, height=256)
    sc, cam = w["scene"], w["cameras"][0]
    p64, p32 = _compare(sc, cam, w["layer_mask"], w["planes"])
    both = (p64["vis"] > 0) & (p32["vis"] > 0)
    # culls agree except where the f64 quantity is on a boundary (none expected here)
    assert np.array_equal(p64["vis"], p32["vis"])
    assert both.sum() > 100
    for k, tol in (("u", 1e-4), ("v", 1e-4), ("depth", 1e-6)):
        assert np.abs(p64[k][both] - p32[k][both]).max() < tol * max(1.0, np.abs(p64[k][both]).max())
    for k in ("A2", "beta", "G2"):
        rel = np.abs(p64[k][both] - p32[k][both]) / np.maximum(np.abs(p64[k][both]), 1e-3)
        assert np.percentile(rel, 99) < 1e-4, k
    assert np.abs(p64["opac"][both] - p32["opac"][both]).max() < 1e-6
    assert np.abs(p64["rgb"][both] - p32["rgb"][both]).max() < 1e-5
    # integer decisions: equal wherever the f64 value is not within 1e-5 of a boundary
    r_exact = 3 * np.sqrt(0.5 * (p64["cov2d"][:, 0] + p64["cov2d"][:, 2]) + np.sqrt(np.maximum(
        0.1, (0.5 * (p64["cov2d"][:, 0] + p64["cov2d"][:, 2])) ** 2 -
        (p64["cov2d"][:, 0] * p64["cov2d"][:, 2] - p64["cov2d"][:, 1] ** 2))))
    near = np.abs(r_exact - np.round(r_exact)) < 1e-5 * np.maximum(1, r_exact)
    ok = both & ~near
    assert np.array_equal(p64["radius"][ok], p32["radius"][ok])
    assert np.array_equal(p64["rect"][ok], p32["rect"][ok])
    # depth keys: the f32 depth is within one unit in the last place of the rounded f64 depth
    d32 = p32["depth_f32"][both]
    d64r = p64["depth"][both].astype(np.float32)
    assert np.abs(d32.view(np.int32).astype(np.int64) - d64r.view(np.int32).astype(np.int64)).max() <= 2


def test_f32_render_close_to_f64_render():
    w = synth.scene_c2(scale=0.005, width=128, height=128)
    sc, cam = w["scene"], w["cameras"][0]
    a = oracle.render(sc, cam, w["layer_mask"], w["planes"], w["bg"], "f64")
    b = oracle.render(sc, cam, w["layer_mask"], w["planes"], w["bg"], "f32")
    mse = ((a["image"] - b["image"]) ** 2).mean()
    assert mse == 0 or 10 * math.log10(1.0 / mse) > 80


def test_f32_half_storage_dequantises_exactly():
    w = synth.scene_c1(scale=0.1)
    sc = w["scene"]
    for kind in ("f16", "bf16"):
        q = synth.from_half_storage(synth.to_half_storage(sc.sh, kind), kind)
        # widening back is exact: re-quantising gives the same bits
        assert np.array_equal(synth.to_half_storage(q, kind), synth.to_half_storage(sc.sh, kind))
        rel = np.abs(q - sc.sh) / np.maximum(np.abs(sc.sh), 1e-3)
        assert rel.max() < (2 ** -10 if kind == "f16" else 2 ** -7)

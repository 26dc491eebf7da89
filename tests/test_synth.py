"""The seeded input generators follow the stated workload recipe: counts and
layers, shell radii and jitter, parameter distributions, cameras, clip planes
and masks; the same seed gives the same arrays; 16-bit storage rounds like an
independent conversion."""
import math

import numpy as np
import pytest
import torch

import synth


def _centre(cam):
    return -(cam.R.astype(np.float64).T @ cam.t.astype(np.float64))


def test_same_seed_same_scene():
    a, b = synth.scene_c2(scale=0.01), synth.scene_c2(scale=0.01)
    for f in ("means", "log_scales", "quats", "opacity_logit", "sh", "layer"):
        assert np.array_equal(getattr(a["scene"], f), getattr(b["scene"], f)), f
    assert a["layer_mask"] == b["layer_mask"]
    assert np.array_equal(a["planes"][0][0], b["planes"][0][0]) and a["planes"][0][1] == b["planes"][0][1]


def test_c2_recipe():
    w = synth.scene_c2()
    sc = w["scene"]
    assert sc.n == 1_200_000 and sc.sh_degree == 3 and sc.sh.shape == (sc.n, 16, 3)
    assert sc.means.dtype == np.float32 and sc.layer.dtype == np.uint8
    counts = np.bincount(sc.layer, minlength=5)
    assert list(counts) == [400_000, 300_000, 250_000, 100_000, 150_000]
    m = sc.means.astype(np.float64) / np.array([1.0, 0.8, 1.25])     # ellipsoid semi-axes (r, 0.8r, 1.25r)
    rad = np.linalg.norm(m, axis=1)
    for L, r in enumerate((0.9, 0.75, 0.5, 0.4, 0.3)):
        x = rad[sc.layer == L] / r
        assert abs(x.mean() - 1.0) < 1e-3 and abs(x.std() - 0.02) < 1e-3, L   # radial jitter N(0, 0.02 r)
    ls = sc.log_scales.astype(np.float64)
    assert abs(ls.mean() + 4.5) < 5e-3 and abs(ls.std() - 0.7) < 5e-3
    assert np.allclose(np.linalg.norm(sc.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert abs(sc.sh.astype(np.float64).std() - 0.2) < 1e-3
    assert 1 <= w["layer_mask"] <= 31
    (nrm, d, bits), = w["planes"]
    assert abs(np.linalg.norm(nrm) - 1.0) < 1e-6 and abs(d) <= 0.3 and bits == 0xFFFFFFFF
    cam, = w["cameras"]
    assert (cam.width, cam.height) == (1024, 1024)
    assert np.allclose(_centre(cam), [0.0, 0.0, 4.0], atol=1e-5)
    assert abs(2 * math.degrees(math.atan(0.5 * cam.width / cam.fx)) - 50.0) < 1e-3   # 50 degree horizontal FoV


def test_c3_recipe():
    w = synth.scene_c3()
    sc, tgt = w["scene"], w["target_scene"]
    assert sc.n == 500_000 and list(np.bincount(sc.layer)) == [200_000, 150_000, 150_000]
    assert len(w["cameras"]) == 8
    for cam in w["cameras"]:
        assert (cam.width, cam.height) == (800, 800)
        assert abs(np.linalg.norm(_centre(cam)) - 4.0) < 1e-5
    ys = sorted(round(float(_centre(c)[1]) / 4.0, 6) for c in w["cameras"])
    assert np.allclose(ys, sorted(1 - 2 * (i + 0.5) / 8 for i in range(8)), atol=1e-6)   # Fibonacci heights
    assert abs((tgt.means - sc.means).astype(np.float64).std() - 0.01) < 1e-4
    assert abs((tgt.sh - sc.sh).astype(np.float64).std() - 0.05) < 1e-4
    assert abs((tgt.opacity_logit - sc.opacity_logit).astype(np.float64).std() - 0.3) < 3e-3


def test_c4_stereo_recipe():
    w = synth.scene_c4(scale=0.01)
    left, right = w["cameras"]
    assert (left.width, left.height) == (2064, 2208)
    assert np.array_equal(left.R, right.R)
    assert abs(np.linalg.norm(_centre(right) - _centre(left)) - 0.064) < 1e-6     # 64 mm eye offset
    assert list(np.bincount(w["scene"].layer)) == [round(2.5 * c * 0.01) for c in synth.scenes.C2_COUNTS]


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_half_storage_rounds_like_torch(kind):
    rng = np.random.default_rng(5)
    a = np.concatenate([rng.normal(0, 3, 20000), rng.normal(0, 1e-3, 2000), [0.0, -0.0, 1.0, 65504.0]])
    a = a.astype(np.float32)
    got = synth.to_half_storage(a, kind)
    t = torch.from_numpy(a)
    if kind == "f16":
        ref = t.to(torch.float16).numpy()
        assert np.array_equal(got.view(np.uint16), ref.view(np.uint16))
    else:
        ref = t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        assert np.array_equal(got, ref)
    back = synth.from_half_storage(got, kind)
    assert np.array_equal(back, t.to(torch.float16 if kind == "f16" else torch.bfloat16).float().numpy())

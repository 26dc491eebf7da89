"""Pins of the oracle's analytic backward (the gradients that drive the layered
training of Sec. 3.2) by central finite differences of its own FP64 forward.

A finite-difference sample is rejected when any discrete decision (cull, tile
rectangle, per-pixel set of blended splats, 0.99 clamp state, stop position)
differs between theta+h and theta-h; such a sample does not have a derivative."""
import math

import numpy as np
import pytest

import oracle
from synth import Scene, look_at_camera
from tests.helpers import make_scene

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _f64_scene(sc):
    return Scene(*(getattr(sc, f).astype(np.float64) for f in FIELDS), sc.layer.copy(), sc.sh_degree)


def _loss_and_sig(sc, cam, w_img, w_a, bg, mask, planes):
    r = oracle.render(sc, cam, layer_mask=mask, planes=planes, bg=bg)
    L = float((w_img * r["image"]).sum() + (w_a * r["alpha"]).sum())
    pre = r["pre"]
    sig = (pre["vis"].tobytes(), pre["rect"].tobytes(), r["dhash"].tobytes())
    return L, sig


def _scene(seed, n=10, deg=3):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.35, 0.35, (n, 3))
    ls = rng.normal(-2.6, 0.35, (n, 3))
    q = rng.standard_normal((n, 4))
    ol = rng.normal(0.3, 1.0, n)
    K = (deg + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, K, 3))
    layer = rng.integers(0, 3, n)
    sc = make_scene(means, ls, q, ol, layer=layer, sh_degree=deg, sh=sh)
    return _f64_scene(sc)


@pytest.mark.parametrize("seed,deg", [(21, 3), (22, 1), (23, 0)])
def test_gradients_match_central_differences(seed, deg):
    sc = _scene(seed, deg=deg)
    cam = look_at_camera((0.3, -0.2, 2.6), width=40, height=32)
    rng = np.random.default_rng(seed + 100)
    bg = np.array([0.3, 0.1, 0.6])
    w_img = rng.standard_normal((3, 32, 40))
    w_a = rng.standard_normal((32, 40))
    planes = [(np.array([0.3, 0.9, 0.3], np.float32) / np.linalg.norm([0.3, 0.9, 0.3]), np.float32(0.25),
               0b010)]
    mask = 0b111
    fwd = oracle.render(sc, cam, layer_mask=mask, planes=planes, bg=bg)
    an = oracle.render_backward(sc, cam, fwd, bg, w_img, w_a)
    vis = np.nonzero(fwd["pre"]["vis"])[0]
    assert vis.size >= 5
    checked = rejected = 0
    for f in FIELDS:
        arr = getattr(sc, f)
        g = an[f]
        scale = np.abs(g).max() + 1e-300
        for i in vis:
            for j in np.ndindex(arr.shape[1:]):
                idx = (i,) + j
                th = arr[idx]
                h = 1e-6 * max(1.0, abs(th))
                arr[idx] = th + h
                Lp, sp = _loss_and_sig(sc, cam, w_img, w_a, bg, mask, planes)
                arr[idx] = th - h
                Lm, sm = _loss_and_sig(sc, cam, w_img, w_a, bg, mask, planes)
                arr[idx] = th
                if sp != sm:
                    rejected += 1
                    continue
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-4 * abs(g[idx]) + 1e-6 * scale + 1e-8, (f, idx, fd, g[idx])
                checked += 1
    assert checked > 0.8 * (checked + rejected)


def test_frozen_layers_get_zero_gradient():
    sc = _scene(24)
    cam = look_at_camera((0.0, 0.0, 2.6), width=32, height=32)
    bg = np.zeros(3)
    fwd = oracle.render(sc, cam, bg=bg)
    w = np.ones((3, 32, 32))
    full = oracle.render_backward(sc, cam, fwd, bg, w)
    part = oracle.render_backward(sc, cam, fwd, bg, w, grad_layer_mask=0b001)
    frozen = sc.layer != 0
    for f in FIELDS:
        assert np.all(part[f][frozen] == 0)
        assert np.array_equal(part[f][~frozen], full[f][~frozen])


def test_contribution_of_a_lone_splat():
    # T = 1 everywhere, so contrib_sum = sum of its alphas and contrib_max = max
    sc = _f64_scene(make_scene([[0.0, 0.0, 0.0]], math.log(0.03), rgb=[0.5, 0.5, 0.5], opacity_logit=0.8))
    cam = look_at_camera((0.0, 0.0, 4.0), width=33, height=33)
    fwd = oracle.render(sc, cam, bg=np.zeros(3))
    cb = oracle.render_backward(sc, cam, fwd, np.zeros(3), np.zeros((3, 33, 33)))
    assert abs(cb["contrib_sum"][0] - fwd["alpha"].sum()) < 1e-12
    assert cb["contrib_max"][0] == fwd["alpha"].max()
    # terms of the sum: the pixels where the closed form o exp(-|d|^2 / (2 s'^2)),
    # s'^2 = (fx s / z0)^2 + 0.3, reaches 1/255 (the 3x3 pixels around the centre)
    o = 1 / (1 + math.exp(-0.8))
    s2 = (cam.fx * 0.03 / 4.0) ** 2 + 0.3
    gy, gx = np.mgrid[0:33, 0:33] + 0.5
    a = o * np.exp(-((gx - 16.5) ** 2 + (gy - 16.5) ** 2) / (2 * s2))
    assert cb["contrib_count"][0] == (a >= 1 / 255).sum() == 9


def test_contribution_of_a_covered_splat():
    # two stacked splats: the far one is weighted by the near one's transmittance
    sc = _f64_scene(make_scene([[0, 0, 0.3], [0, 0, -0.3]], math.log(0.05), rgb=[0.5, 0.5, 0.5],
                               opacity_logit=[1.0, 1.0]))
    cam = look_at_camera((0.0, 0.0, 4.0), width=33, height=33)
    fwd = oracle.render(sc, cam, bg=np.zeros(3))
    cb = oracle.render_backward(sc, cam, fwd, np.zeros(3), np.zeros((3, 33, 33)))
    o = 1 / (1 + math.exp(-1.0))
    assert abs(cb["contrib_max"][0] - o) < 1e-12
    assert abs(cb["contrib_max"][1] - o * (1 - o)) < 1e-12
    # the near splat is larger on screen, so it is blended wherever the far one
    # is: the terms are the pixels with any blend plus those whose last blended
    # list entry is the far splat (n_contrib = 2)
    assert cb["contrib_count"][0] > 0 and cb["contrib_count"][1] > 0
    assert cb["contrib_count"].sum() == ((fwd["alpha"] > 0).sum() + (fwd["ncontrib"] >= 2).sum())


def test_gradients_through_clamps():
    # opaque splats (alpha clamped at 0.99 near their centres), colours clamped at
    # zero, and large splats centred beyond 1.3x the half field of view whose
    # Jacobian is taken on the clamped ray
    rng = np.random.default_rng(25)
    n = 9
    means = rng.uniform(-0.3, 0.3, (n, 3))
    means[6:, 0] = [1.9, -1.95, 2.1]           # beyond the frustum clamp at depth ~2.6
    ls = rng.normal(-2.4, 0.3, (n, 3))
    ls[6:] = np.log(0.5)
    q = rng.standard_normal((n, 4))
    ol = rng.normal(4.0, 1.5, n)
    sh = rng.normal(0.0, 0.3, (n, 4, 3))
    sh[:3, 0, 0] = -3.0                        # red channel clamped at zero
    sc = _f64_scene(make_scene(means, ls, q, ol, sh_degree=1, sh=sh))
    cam = look_at_camera((0.0, 0.0, 2.6), width=48, height=40)
    w_img = rng.standard_normal((3, 40, 48))
    bg = np.array([0.2, 0.2, 0.2])
    fwd = oracle.render(sc, cam, bg=bg)
    pre = fwd["pre"]
    lim = 1.3 * 0.5 * 48 / cam.fx
    pz = sc.means @ cam.R.T.astype(np.float64) + cam.t
    assert np.any((np.abs(pz[:, 0] / pz[:, 2]) > lim) & (pre["vis"] > 0)), "no clamped-Jacobian splat visible"
    assert np.any(fwd["alpha"] > 0.99 - 1e-12)
    an = oracle.render_backward(sc, cam, fwd, bg, w_img)
    checked = 0
    for f in FIELDS:
        arr, g = getattr(sc, f), an[f]
        scale = np.abs(g).max() + 1e-300
        for i in np.nonzero(pre["vis"])[0]:
            for j in np.ndindex(arr.shape[1:]):
                idx = (i,) + j
                th = arr[idx]
                h = 1e-6 * max(1.0, abs(th))
                arr[idx] = th + h
                Lp, sp = _loss_and_sig(sc, cam, w_img, 0.0, bg, 0xFFFFFFFF, [])
                arr[idx] = th - h
                Lm, sm = _loss_and_sig(sc, cam, w_img, 0.0, bg, 0xFFFFFFFF, [])
                arr[idx] = th
                if sp != sm:
                    continue
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-4 * abs(g[idx]) + 1e-6 * scale + 1e-8, (f, idx, fd, g[idx])
                checked += 1
    assert checked > 150

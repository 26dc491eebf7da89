"""GPU parity of the forward path (S1 preprocess, S2 binning + sorts, S3
compositing) against the FP64 oracle, called through the C ABI.

Bars: bit-exact records' integer decisions, tile ids and order; colours within
1e-5 absolute of the oracle composited from the same single-precision
projection (fragile threshold decisions may take either side); PSNR >= 50 dB
against the end-to-end FP64 render."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (compare_image, compare_lists, compare_records, dequantised, gpu_render, oracle_stage,
                            psnr, read_ws)
from tests.helpers import axis_camera, make_scene, random_small_scene

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _workloads():
    w1 = synth.scene_c1()
    rng = np.random.default_rng(77)
    sc2 = synth.shell_scene(rng, [6000, 4500, 3750, 1500, 2250], synth.scenes.C2_RADII)
    cam2 = synth.look_at_camera((0.3, -0.2, 3.2), fov_x_deg=50.0, width=200, height=152)
    planes2 = synth.random_clip_planes(rng, 1)
    return {
        "c1": (w1["scene"], w1["cameras"][0], w1["layer_mask"], w1["planes"], (0.0, 0.0, 0.0)),
        "shells_ragged": (sc2, cam2, 0b10111, planes2, (0.2, 0.3, 0.4)),
    }


WL = _workloads()


@pytest.mark.parametrize("name", list(WL))
def test_forward_parity(name):
    sc, cam, mask, planes, bg = WL[name]
    ds, rast, img, al = gpu_render(sc, cam, mask, planes, bg)
    ws = read_ws(rast)
    assert ws["status"].error == 0
    pre, ranges, lst, co = oracle_stage(sc, cam, mask, planes, bg)
    compare_records(ws, pre)
    compare_lists(ws, ranges, lst)
    st = compare_image(img.cpu().numpy(), al.cpu().numpy(), ws["n_contrib"].astype(np.int64), co, TOL)
    print(name, st)
    assert st["n_bad"] == 0, st
    assert st["n_multi"] <= 0.001 * sc.n
    full = oracle.render(sc, cam, mask, planes, bg, "f64")
    assert psnr(img.cpu().numpy(), full["image"]) >= 50.0


@pytest.mark.parametrize("kind", [("f16", "f32"), ("bf16", "bf16"), ("f16", "f16")])
def test_half_storage_records_and_image(kind):
    sh_dt, sr_dt = kind
    sc, cam, mask, planes, bg = WL["shells_ragged"]
    ds, rast, img, al = gpu_render(sc, cam, mask, planes, bg, sh_dtype=sh_dt, sr_dtype=sr_dt)
    ws = read_ws(rast)
    sq = dequantised(sc, sh_dt, sr_dt)
    pre, ranges, lst, co = oracle_stage(sq, cam, mask, planes, bg)
    compare_records(ws, pre)
    compare_lists(ws, ranges, lst)
    st = compare_image(img.cpu().numpy(), al.cpu().numpy(), ws["n_contrib"].astype(np.int64), co, TOL)
    assert st["n_bad"] == 0, st
    # precision cost of 16-bit storage against the FP64 render of the FP32 master scene
    ref = oracle.render(sc, cam, mask, planes, bg, "f64")
    print(kind, "PSNR vs FP32 master", psnr(img.cpu().numpy(), ref["image"]))


def test_mask_zero_is_background():
    sc, cam, _, _, _ = WL["c1"]
    bg = (0.25, 0.5, 0.75)
    _, rast, img, al = gpu_render(sc, cam, 0, (), bg)
    want = torch.tensor(bg, device=img.device).view(3, 1, 1).expand_as(img)
    assert torch.equal(img, want)
    assert torch.all(al == 0)
    assert read_ws(rast)["D"] == 0


def test_empty_scene():
    sc = make_scene(np.zeros((0, 3)), np.zeros((0, 3)))
    cam = axis_camera(4.0, 40, 24)
    _, rast, img, al = gpu_render(sc, cam, bg=(0.1, 0.2, 0.3))
    assert torch.allclose(img[0], torch.full_like(img[0], 0.1))
    assert torch.all(al == 0)


def test_single_splat_closed_form():
    z0, s, o = 4.0, 0.02, 0.6
    cam = axis_camera(z0, 33, 33)
    sc = make_scene([[0, 0, 0]], math.log(s), rgb=[0.9, 0.5, 0.25], opacity_logit=math.log(o / (1 - o)))
    _, rast, img, al = gpu_render(sc, cam, bg=(0.1, 0.2, 0.3))
    o = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    rgb = sc.sh[0, 0].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    want = o * rgb + (1 - o) * np.array([0.1, 0.2, 0.3])
    assert np.abs(img[:, 16, 16].cpu().numpy() - want).max() < 1e-6


@pytest.mark.parametrize("mask", [0b00001, 0b00110, 0b11010])
def test_masking_equals_deleting_on_gpu(mask):
    sc, cam, _, _, bg = WL["shells_ragged"]
    _, _, a, aa = gpu_render(sc, cam, mask, (), bg)
    keep = ((mask >> sc.layer.astype(np.int64)) & 1).astype(bool)
    _, _, b, bb = gpu_render(sc.subset(keep), cam, 0xFFFFFFFF, (), bg)
    assert torch.equal(a, b) and torch.equal(aa, bb)


def test_clipping_equals_deleting_on_gpu():
    sc, cam, _, _, bg = WL["shells_ragged"]
    rng = np.random.default_rng(5)
    planes = synth.random_clip_planes(rng, 2, 0.3, layer_bits=0b00111)
    _, rast, a, aa = gpu_render(sc, cam, 0xFFFFFFFF, planes, bg)
    pre = oracle.preprocess(sc, cam, 0xFFFFFFFF, planes, "f32")
    pre_all = oracle.preprocess(sc, cam, 0xFFFFFFFF, (), "f32")
    keep = ~((pre_all["vis"] > 0) & (pre["vis"] == 0))
    _, _, b, bb = gpu_render(sc.subset(keep), cam, 0xFFFFFFFF, (), bg)
    assert torch.equal(a, b) and torch.equal(aa, bb)


def test_overflow_reports_and_recovers():
    sc, cam, mask, planes, bg = WL["shells_ragged"]
    _, rast, img_small, _ = gpu_render(sc, cam, mask, planes, bg, cap=1000, check=False)
    st = rast.status()
    assert st.error == 2 and st.n_dup > 1000 and st.dup_capacity >= 1000
    _, rast2, img_ok, _ = gpu_render(sc, cam, mask, planes, bg, cap=1000, check=True)
    assert rast2.status().error == 0 and rast2.dup_capacity > 1000
    _, _, img_ref, _ = gpu_render(sc, cam, mask, planes, bg)
    assert torch.equal(img_ok, img_ref)


def test_stereo_eyes_equal_mono_renders():
    w = synth.scene_c4(scale=0.002, width=96, height=104)
    sc = w["scene"]
    for cam in w["cameras"]:
        _, rast, img, al = gpu_render(sc, cam, w["layer_mask"], w["planes"], (0, 0, 0))
        pre, ranges, lst, co = oracle_stage(sc, cam, w["layer_mask"], w["planes"], (0, 0, 0))
        nc = read_ws(rast)["n_contrib"].astype(np.int64)
        st = compare_image(img.cpu().numpy(), al.cpu().numpy(), nc, co, TOL)
        assert st["n_bad"] == 0, st


def test_repeated_renders_are_deterministic():
    sc, cam, mask, planes, bg = WL["shells_ragged"]
    ds, rast, a, _ = gpu_render(sc, cam, mask, planes, bg)
    b, _ = rast.render(ds, cam, mask, planes, bg)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def _batch_views():
    """Mixed views: two scenes, four sizes, masks, planes, backgrounds, a stereo pair."""
    sc1, cam1, m1, p1, bg1 = WL["c1"]
    sc2, cam2, m2, p2, bg2 = WL["shells_ragged"]
    w4 = synth.scene_c4(scale=0.002, width=96, height=104)
    rng = np.random.default_rng(5)
    views = [(sc1, cam1, m1, p1, bg1), (sc2, cam2, m2, p2, bg2), (sc2, cam2, 0b00011, (), (1.0, 1.0, 1.0)),
             (sc1, synth.look_at_camera((0.0, 4.0, 0.5), width=72, height=40), 0b01, (), (0.1, 0.2, 0.3)),
             (sc2, cam2, 0, (), (0.5, 0.5, 0.5))]
    for cam in w4["cameras"]:
        views.append((w4["scene"], cam, w4["layer_mask"], w4["planes"], (0.0, 0.0, 0.0)))
    for k in range(3):
        views.append((sc2, synth.look_at_camera(3.0 * rng.standard_normal(3) + 0.1, width=48 + 16 * k, height=33),
                      int(rng.integers(1, 32)), tuple(synth.random_clip_planes(rng, 2)), (0.0, 0.0, 0.0)))
    return views


def test_render_batch_equals_single_renders():
    """gs_render_batch composites all views in one launch; every view's image,
    alpha and forward state equal those of its own gs_render call."""
    from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
    views = _batch_views()
    dss = {}
    singles, items, rasts = [], [], []
    for sc, cam, m, p, bg in views:
        ds = dss.setdefault(id(sc), DeviceScene.from_host(sc))
        r0 = Rasterizer(sc.n, cam.width, cam.height)
        a_img, a_al = r0.render(ds, cam, m, p, bg)
        singles.append((a_img, a_al, read_ws(r0)))
        r1 = Rasterizer(sc.n, cam.width, cam.height)
        rasts.append(r1)
        img = torch.full((3, cam.height, cam.width), float("nan"), device="cuda")
        al = torch.full((cam.height, cam.width), float("nan"), device="cuda")
        items.append(dict(scene=ds.c_struct(), camera=_lib.make_camera(cam), layer_mask=m, planes=list(p), bg=bg,
                          workspace=r1.workspace, ws_bytes=r1.ws_bytes, image=img, alpha=al))
    _lib.gs_render_batch(items, 0)
    torch.cuda.synchronize()
    for k, (it, r1, (a_img, a_al, wa)) in enumerate(zip(items, rasts, singles)):
        wb = read_ws(r1)
        assert wb["status"].error == 0, k
        assert torch.equal(it["image"], a_img), k
        assert torch.equal(it["alpha"], a_al), k
        assert np.array_equal(wa["n_contrib"], wb["n_contrib"]), k
        assert np.array_equal(wa["t_final"], wb["t_final"]), k


def test_render_batch_limits_and_overflow_isolation():
    """More than GS_MAX_BATCH views is refused; a view that overflows its pair
    capacity reports it in its own status word and leaves the others intact."""
    from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
    sc, cam, m, p, bg = WL["shells_ragged"]
    ds = DeviceScene.from_host(sc)
    ref_img, _ = Rasterizer(sc.n, cam.width, cam.height).render(ds, cam, m, p, bg)

    def item(r):
        return dict(scene=ds.c_struct(), camera=_lib.make_camera(cam), layer_mask=m, planes=list(p), bg=bg,
                    workspace=r.workspace, ws_bytes=r.ws_bytes,
                    image=torch.empty((3, cam.height, cam.width), device="cuda"), alpha=None)

    r_ok = Rasterizer(sc.n, cam.width, cam.height)
    with pytest.raises(ValueError):
        _lib.gs_render_batch([item(r_ok)] * (_lib.GS_MAX_BATCH + 1), 0)
    with pytest.raises(_lib.GsError):
        _lib.gs_render_batch([item(r_ok), item(r_ok)], 0)   # one workspace shared by two views
    r_small = Rasterizer(sc.n, cam.width, cam.height, dup_capacity=1000)
    its = [item(r_small), item(r_ok)]
    _lib.gs_render_batch(its, 0)
    torch.cuda.synchronize()
    assert r_small.status().error == _lib.GS_ERR_WORKSPACE
    assert r_ok.status().error == 0
    assert torch.equal(its[1]["image"], ref_img)


def test_blended_pair_count():
    """The status word's blended-pair count equals the number of (pixel,
    Gaussian) pairs the oracle blends (up to one per fragile pixel)."""
    sc, cam, mask, planes, bg = WL["shells_ragged"]
    _, rast, img, al = gpu_render(sc, cam, mask, planes, bg)
    st = rast.status()
    pre, ranges, lst, co = oracle_stage(sc, cam, mask, planes, bg)
    W, H = cam.width, cam.height
    Tx = (W + 15) // 16
    count = 0
    for y in range(H):
        for x in range(W):
            t = (y // 16) * Tx + x // 16
            ids = lst[ranges[t, 0]:ranges[t, 0] + co["ncontrib"][y, x]]
            if ids.size == 0:
                continue
            dx = x + 0.5 - pre["u"][ids]
            dy = y + 0.5 - pre["v"][ids]
            p = dx + pre["beta"][ids] * dy
            a = np.minimum(0.99, pre["opac"][ids] * np.exp2(pre["A2"][ids] * p * p + pre["G2"][ids] * dy * dy))
            count += int((a >= 1.0 / 255.0).sum())
    assert abs(int(st.n_blended) - count) <= int((co["fragile"] > 0).sum()), (st.n_blended, count)

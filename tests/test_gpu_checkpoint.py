"""Saving and loading on the GPU: device scenes in every storage precision
(FP32, FP16/BF16, the SH codebook) come back byte for byte and render the
same image; layers merged on the device render as the cloud they came from;
and a Trainer restored from its checkpoint continues the saved run: the
restored state is identical, and its next step agrees with the original
trainer's next step up to the rounding order of the gradient atomics."""
import numpy as np
import pytest
import torch

import synth
from paper_2410_16978_gb300 import DeviceScene, Rasterizer, checkpoint as ck
from paper_2410_16978_gb300.train import TrainConfig, Trainer

pytestmark = pytest.mark.gpu
FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh", "layer")


def _bytes(t):
    return t.contiguous().view(torch.uint8)


def _render(ds, cam, mask, planes):
    r = Rasterizer(ds.n, cam.width, cam.height)
    img, al = r.render(ds, cam, mask, planes, (0.1, 0.2, 0.3), check=True)
    torch.cuda.synchronize()
    return img, al


@pytest.mark.parametrize("shdt,srdt", [("f32", "f32"), ("f16", "bf16"), ("bf16", "f16")])
def test_device_scene_round_trip(shdt, srdt, tmp_path):
    w = synth.scene_c2(scale=0.02, width=256, height=256)
    ds = DeviceScene.from_host(w["scene"], sh_dtype=shdt, sr_dtype=srdt)
    p = str(tmp_path / "s.npz")
    ck.save_scene(p, ds)
    back = ck.load_scene(p, device="cuda")
    assert (back.sh_dtype, back.sr_dtype, back.sh_degree) == (shdt, srdt, 3)
    for f in FIELDS:
        a, b = getattr(ds, f), getattr(back, f)
        assert a.dtype == b.dtype and a.shape == b.shape and torch.equal(_bytes(a), _bytes(b)), f
    cam = w["cameras"][0]
    for x, y in zip(_render(ds, cam, w["layer_mask"], w["planes"]), _render(back, cam, w["layer_mask"], w["planes"])):
        assert torch.equal(x, y)


def test_codebook_scene_round_trip(tmp_path):
    from paper_2410_16978_gb300.codebook import build_sh_codebook
    w = synth.scene_c2(scale=0.01, width=192, height=192)
    ds = DeviceScene.from_host(w["scene"])
    cb, _, _ = build_sh_codebook(ds, size=256, iters=2, seed=1)
    p = str(tmp_path / "cb.npz")
    ck.save_scene(p, cb)
    back = ck.load_scene(p, device="cuda")
    assert back.sh_dtype == "cb"
    for f in FIELDS + ("sh_index", "sh_table"):
        assert torch.equal(_bytes(getattr(cb, f)), _bytes(getattr(back, f))), f
    cam = w["cameras"][0]
    for x, y in zip(_render(cb, cam, w["layer_mask"], w["planes"]), _render(back, cam, w["layer_mask"], w["planes"])):
        assert torch.equal(x, y)


def test_layers_merged_on_the_device_render_as_the_whole_cloud():
    w = synth.scene_c2(scale=0.02, width=256, height=256)
    sc = w["scene"]
    parts = [DeviceScene.from_host(sc.subset(np.nonzero(sc.layer == L)[0])) for L in range(5)]
    merged = ck.merge_layers(parts)
    whole = DeviceScene.from_host(sc)
    for f in FIELDS:
        assert torch.equal(_bytes(getattr(merged, f)), _bytes(getattr(whole, f))), f
    cam = w["cameras"][0]
    for x, y in zip(_render(merged, cam, w["layer_mask"], w["planes"]),
                    _render(whole, cam, w["layer_mask"], w["planes"])):
        assert torch.equal(x, y)


def test_trainer_resumes_from_checkpoint(tmp_path):
    w = synth.scene_c3(scale=0.02, width=128, height=128)
    cams = w["cameras"]
    tgt = DeviceScene.from_host(w["target_scene"])
    targets = []
    for cam in cams[:3]:
        img, al = _render(tgt, cam, w["layer_mask"], ())
        targets.append((img.clone(), al.clone()))
    cfg = TrainConfig(w_alpha=0.8, train_layer_mask=0b011, activity_prune=True, activity_interval=1000)
    tr = Trainer(DeviceScene.from_host(w["scene"]), cams, cfg)
    rng = np.random.default_rng(0)
    bgs = [tuple(float(v) for v in rng.uniform(0, 1, 3)) for _ in range(5)]
    for k in range(3):
        tr.step(k, *targets[k], bgs[k])
    torch.cuda.synchronize()
    p = str(tmp_path / "trainer.npz")
    ck.save_trainer(p, tr)
    back = ck.load_trainer(p, cams)
    assert back.t == tr.t == 3 and back.activity_samples == tr.activity_samples == 3
    assert back.activity_threshold == tr.activity_threshold and back.cfg == tr.cfg
    for f in FIELDS:
        assert torch.equal(_bytes(getattr(tr.scene, f)), _bytes(getattr(back.scene, f))), f
    for a, b in zip(tr.m + tr.v + [tr.contrib_max, tr.contrib_sum, tr.activity],
                    back.m + back.v + [back.contrib_max, back.contrib_sum, back.activity]):
        assert torch.equal(a, b)
    # the next step of both: the same update up to the rounding order of float atomics
    tr.step(0, *targets[0], bgs[3])
    back.step(0, *targets[0], bgs[3])
    torch.cuda.synchronize()
    for f, lr in zip(FIELDS[:5], cfg.lr):
        a, b = getattr(tr.scene, f).detach(), getattr(back.scene, f).detach()
        assert float((a - b).abs().max()) <= 1e-3 * lr, f     # Adam moves each parameter by about lr at most
    frozen = (back.scene.layer == 2)
    assert torch.equal(back.scene.means.detach()[frozen], DeviceScene.from_host(w["scene"]).means[frozen])

"""Precision variants of the mixed-precision workload (3M Gaussians in 5
layers, stereo 2 x 2064x2208): SH and log-scale/rotation stored in FP16 or
BF16, means, opacity, compositing and transmittance in FP32.  Each variant's
render is compared with the end-to-end FP64 oracle render of the FP32 master
scene on sampled pixels (uniform plus whole rows through the centre), and the
PSNR and maximum absolute error are printed per eye and variant.

Bars: every variant reaches the method's acceptance bar of 50 dB, and each
has its own PSNR floor and maximum absolute error: the values measured on a
GB300 (FP32 121.9 / 100.5 dB and 2.0e-4 / 2.3e-3; FP16 SH + FP16 scale/rot
76.6 / 76.7 dB and 4.2e-3 / 3.8e-3; FP16 + BF16 62.8 / 62.7 dB and 7.7e-3 /
7.0e-3; BF16 + FP16 75.3 / 75.3 dB and 4.2e-3 / 3.8e-3; BF16 + BF16 62.6 /
62.6 dB and 7.7e-3 / 7.0e-3, left / right eye) less a margin of 3 dB, and
twice the measured maximum error, rounded up.  The 16-bit errors are the
storage rounding; the FP32 maximum comes from pixels where a single-precision
threshold decision differs from the FP64 one."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import gpu_render, psnr

pytestmark = pytest.mark.gpu

VARIANTS = [("f32", "f32"), ("f16", "f16"), ("f16", "bf16"), ("bf16", "f16"), ("bf16", "bf16")]
# (PSNR floor in dB, max |error|) per (SH storage, scale/rotation storage)
BARS = {("f32", "f32"): (97.0, 5e-3), ("f16", "f16"): (73.5, 1e-2), ("f16", "bf16"): (59.5, 2e-2),
        ("bf16", "f16"): (72.0, 1e-2), ("bf16", "bf16"): (59.5, 2e-2)}


@pytest.fixture(scope="module")
def c4_reference():
    w = synth.scene_c4()
    sc = w["scene"]
    out = []
    rng = np.random.default_rng(44)
    for cam in w["cameras"]:
        W, H = cam.width, cam.height
        xs = rng.integers(0, W, 8192)
        ys = rng.integers(0, H, 8192)
        rows = np.arange(H // 2 - 8, H // 2 + 8)
        gx, gy = np.meshgrid(np.arange(W), rows)
        xs = np.concatenate([xs, gx.ravel()]).astype(np.int32)
        ys = np.concatenate([ys, gy.ravel()]).astype(np.int32)
        pre = oracle.preprocess(sc, cam, w["layer_mask"], w["planes"], "f64")
        ranges, lst = oracle.bin_tiles(pre)
        cp = oracle.composite_pixels(pre, ranges, lst, xs, ys, (0.0, 0.0, 0.0))
        out.append((cam, xs, ys, cp))
    return w, out


@pytest.mark.parametrize("shdt,srdt", VARIANTS)
def test_precision_variant_against_fp64(c4_reference, shdt, srdt):
    w, eyes = c4_reference
    res = []
    for eye, (cam, xs, ys, cp) in enumerate(eyes):
        _, _, img, al = gpu_render(w["scene"], cam, w["layer_mask"], w["planes"], (0.0, 0.0, 0.0), shdt, srdt)
        g = img.cpu().numpy()[:, ys, xs].T.astype(np.float64)
        ref = cp["rgb"]
        assert np.isfinite(g).all()
        err = np.abs(g - ref).max()
        p = psnr(g, ref)
        res.append((eye, p, err))
        floor, max_err = BARS[(shdt, srdt)]
        assert p >= max(50.0, floor), (eye, p)
        assert err <= max_err, (eye, err)
    print("precision SH %s, scale/rot %s:" % (shdt, srdt),
          "; ".join("eye %d PSNR %.2f dB max|err| %.3g" % r for r in res))

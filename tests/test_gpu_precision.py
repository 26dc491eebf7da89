"""Precision variants of the mixed-precision workload (3M Gaussians in 5
layers, stereo 2 x 2064x2208): SH and log-scale/rotation stored in FP16 or
BF16, means, opacity, compositing and transmittance in FP32.  Each variant's
render is compared with the end-to-end FP64 oracle render of the FP32 master
scene on sampled pixels (uniform plus whole rows through the centre), and the
PSNR and maximum absolute error are printed per eye and variant.

Bars: FP32 storage >= 50 dB (the acceptance bar of the method); every
16-bit variant stays finite and within 1e-1 absolute (its error is the
storage rounding, reported, not a defect)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import gpu_render, psnr

pytestmark = pytest.mark.gpu

VARIANTS = [("f32", "f32"), ("f16", "f16"), ("f16", "bf16"), ("bf16", "f16"), ("bf16", "bf16")]


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
        if (shdt, srdt) == ("f32", "f32"):
            assert p >= 50.0, (eye, p)
        assert err <= 1e-1, (eye, err)
    print("precision SH %s, scale/rot %s:" % (shdt, srdt),
          "; ".join("eye %d PSNR %.2f dB max|err| %.3g" % r for r in res))

"""SH codebook (Sec. 3.3, K-means across layers) on the GPU.

* k-means assignment: every point's chosen centroid is a nearest one (FP64
  distances, within single-precision rounding); several may be nearest, so
  the choice itself is not compared.
* k-means update: the mean of each cluster's points (FP64) within 1e-5.
* rendering from codebook storage: records bit-exact and pixels within 1e-5
  of the oracle's render of the dequantised scene, with a codebook built on
  the host (oracle k-means), so no oracle input comes from the GPU.
* the product builder: its codebook scene against the float32-SH render."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import codebook as OCB
from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
from paper_2410_16978_gb300.codebook import build_sh_codebook
from tests.gpu_util import compare_image, compare_records, gpu_render, oracle_stage, psnr, read_ws

pytestmark = pytest.mark.gpu


def test_kmeans_assign_picks_a_nearest_centroid():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5000, 45)).astype(np.float32)
    c = rng.standard_normal((300, 45)).astype(np.float32)
    a = torch.empty(5000, dtype=torch.int32, device="cuda")
    _lib.gs_kmeans_assign(torch.from_numpy(x).cuda(), 5000, 45, 45, torch.from_numpy(c).cuda(), 300, a, 0)
    torch.cuda.synchronize()
    got = a.cpu().numpy().astype(np.int64)
    d_got = OCB.sq_dist(x, c, got)
    d_min = OCB.sq_dist(x, c, OCB.kmeans_assign(x, c))
    assert np.all(d_got <= d_min * (1 + 1e-5) + 1e-6)


def test_kmeans_assign_strided_points_and_update_mean():
    rng = np.random.default_rng(1)
    n, dim, stride, k = 4000, 9, 12, 50
    rows = rng.standard_normal((n, stride)).astype(np.float32)
    pts = rows[:, 3:3 + dim]
    c0 = rng.standard_normal((k, dim)).astype(np.float32)
    R = torch.from_numpy(rows).cuda()
    C = torch.from_numpy(c0).cuda()
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    _lib.gs_kmeans_assign(R.data_ptr() + 12, n, dim, stride, C, k, a, 0)
    torch.cuda.synchronize()
    got = a.cpu().numpy().astype(np.int64)
    assert np.all(OCB.sq_dist(pts, c0, got) <= OCB.sq_dist(pts, c0, OCB.kmeans_assign(pts, c0)) * (1 + 1e-5) + 1e-6)
    # update with a host-made assignment (two clusters left empty)
    assign = rng.integers(0, k - 2, n).astype(np.int32)
    sb = _lib.gs_kmeans_scratch_size(k, dim)
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    _lib.gs_kmeans_update(R.data_ptr() + 12, n, dim, stride, torch.from_numpy(assign).cuda(), k, C, scratch, sb, 0)
    torch.cuda.synchronize()
    want = OCB.kmeans_update(pts, assign, c0)
    assert np.abs(C.cpu().numpy() - want).max() <= 1e-5 * max(1.0, np.abs(want).max())
    assert np.array_equal(C.cpu().numpy()[k - 2:], c0[k - 2:])          # empty clusters keep their centroid


def _host_codebook(sc, k=64, iters=3, seed=2):
    """Codebook storage made on the host with the oracle's k-means."""
    n, K = sc.n, (sc.sh_degree + 1) ** 2
    rest = sc.sh[:, 1:, :].reshape(n, -1).astype(np.float64)
    rng = np.random.default_rng(seed)
    c = rest[rng.choice(n, k, replace=False)]
    for _ in range(iters):
        a = OCB.kmeans_assign(rest, c)
        c = OCB.kmeans_update(rest, a, c)
    a = OCB.kmeans_assign(rest, c)
    R = (3 * (K - 1) + 7) // 8 * 8
    table = np.zeros((k, R), np.float16)
    table[:, :3 * (K - 1)] = c.astype(np.float16)
    dc = sc.sh[:, 0, :].astype(np.float32)
    return dc, a.astype(np.uint16), table


@pytest.mark.parametrize("deg", [1, 3])
def test_codebook_render_matches_oracle(deg):
    rng = np.random.default_rng(3 + deg)
    sc = synth.shell_scene(rng, [3000, 2000], (0.8, 0.45), sh_degree=deg)
    cam = synth.look_at_camera((0.4, -0.3, 3.3), width=120, height=88)
    dc, idx, table = _host_codebook(sc)
    sq = sc.copy()
    sq.sh = OCB.dequantise(dc, table, idx.astype(np.int64), (deg + 1) ** 2).astype(np.float32)
    base = DeviceScene.from_host(sc)
    cbs = DeviceScene(base.means, base.log_scales, base.quats, base.opacity_logit, torch.from_numpy(dc).cuda(),
                      base.layer, deg, "cb", "f32", sh_index=torch.from_numpy(idx.view(np.int16)).cuda(),
                      sh_table=torch.from_numpy(table).cuda())
    r = Rasterizer(sc.n, cam.width, cam.height)
    img, al = r.render(cbs, cam, 0b11, (), (0.1, 0.2, 0.3))
    torch.cuda.synchronize()
    ws = read_ws(r)
    pre, ranges, lst, co = oracle_stage(sq, cam, 0b11, (), (0.1, 0.2, 0.3))
    compare_records(ws, pre)
    st = compare_image(img.cpu().numpy(), al.cpu().numpy(), ws["n_contrib"].astype(np.int64), co, 1e-5)
    assert st["n_bad"] == 0, st
    # backward refuses codebook storage (render only)
    with pytest.raises(_lib.GsError):
        r.backward(cbs, cam, (0.1, 0.2, 0.3), torch.zeros((3, cam.height, cam.width), device="cuda"))


def test_builder_quality_on_the_layered_scene():
    """1.2M-Gaussian layered scene: a 16k-entry codebook trained on 200k
    Gaussians; printed PSNR of the codebook render against the float32-SH
    render, and the SH bytes per Gaussian before and after."""
    w = synth.scene_c2()
    sc, cam = w["scene"], w["cameras"][0]
    ds = DeviceScene.from_host(sc)
    cbs, cent, assign = build_sh_codebook(ds, size=16384, iters=6, sample=200_000, seed=1)
    torch.cuda.synchronize()
    assert int(assign.max()) < 16384 and cbs.sh_table.shape == (16384, 48)
    bg = tuple(float(v) for v in w["bg"])
    _, _, ref, _ = gpu_render(sc, cam, w["layer_mask"], w["planes"], bg)
    r = Rasterizer(sc.n, cam.width, cam.height)
    img, _ = r.render(cbs, cam, w["layer_mask"], w["planes"], bg)
    torch.cuda.synchronize()
    p = psnr(img.cpu().numpy(), ref.cpu().numpy())
    print("codebook 16384 x 45 (FP16) on 1.2M Gaussians: PSNR vs FP32 SH %.2f dB, max |diff| %.3g; SH bytes per "
          "Gaussian 192 -> 14 (+%.1f MB table)" % (p, float((img - ref).abs().max()), 16384 * 96 / 1e6))
    assert p > 30.0

"""Helpers for the GPU tests: run the CUDA path through the C ABI and read the
intermediate workspace regions back to the host."""
import math

import numpy as np
import torch

import oracle
from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
from synth import Scene, from_half_storage, to_half_storage

REC_FIELDS = ("u", "v", "A2", "beta", "G2", "opac")


def gpu_render(scene, cam, mask=0xFFFFFFFF, planes=(), bg=(0.0, 0.0, 0.0), sh_dtype="f32", sr_dtype="f32",
               cap=None, check=True):
    ds = DeviceScene.from_host(scene, sh_dtype=sh_dtype, sr_dtype=sr_dtype)
    rast = Rasterizer(scene.n, cam.width, cam.height, dup_capacity=cap)
    img, al = rast.render(ds, cam, mask, planes, bg, check=check)
    torch.cuda.synchronize()
    return ds, rast, img, al


def read_ws(rast):
    n, W, H = rast.n, rast.width, rast.height
    lay = _lib.gs_workspace_layout(n, W, H, rast.ws_bytes)
    st = rast.status()
    ws = rast.workspace.cpu().numpy()
    Tn = math.ceil(W / 16) * math.ceil(H / 16)
    D = int(min(st.n_dup, lay["dup_capacity"]))

    def region(key, count, dtype):
        nbytes = count * np.dtype(dtype).itemsize
        return ws[lay[key]:lay[key] + nbytes].view(dtype)

    rec = region("rec", 12 * n, np.float32).reshape(n, 12)
    out = dict(status=st, rec=rec, tiles=region("tiles", n, np.uint32), depth=region("depth", n, np.uint32),
               list=region("list", D, np.uint32),
               ranges=region("ranges", 2 * Tn, np.uint32).reshape(Tn, 2),
               t_final=region("t_final", W * H, np.float32).reshape(H, W),
               n_contrib=region("n_contrib", W * H, np.uint32).reshape(H, W), D=D)
    r10 = rec[:, 10].view(np.uint32)
    r11 = rec[:, 11].view(np.uint32)
    out["rect"] = np.stack([r10 & 0xFFFF, r10 >> 16, r11 & 0xFFFF, r11 >> 16], 1).astype(np.int32)
    return out


def dequantised(scene, sh_dtype="f32", sr_dtype="f32"):
    """The float32 values the GPU sees when the scene is stored in 16 bits."""
    sc = scene.copy()
    if sh_dtype != "f32":
        sc.sh = from_half_storage(to_half_storage(sc.sh, sh_dtype), sh_dtype)
    if sr_dtype != "f32":
        sc.log_scales = from_half_storage(to_half_storage(sc.log_scales, sr_dtype), sr_dtype)
        sc.quats = from_half_storage(to_half_storage(sc.quats, sr_dtype), sr_dtype)
    return sc


def f64_scene(sc):
    return Scene(sc.means.astype(np.float64), sc.log_scales.astype(np.float64), sc.quats.astype(np.float64),
                 sc.opacity_logit.astype(np.float64), sc.sh.astype(np.float64), sc.layer.copy(), sc.sh_degree)


def compare_records(ws, pre32):
    """Bit-exact comparison of the GPU records with the oracle's single-precision path."""
    vis_gpu = ws["tiles"] > 0
    vis_or = pre32["vis"] > 0
    assert np.array_equal(vis_gpu, vis_or), "visibility differs at %s" % np.nonzero(vis_gpu != vis_or)[0][:10]
    assert np.array_equal(ws["tiles"][vis_or].astype(np.int64), pre32["tiles"][vis_or])
    assert np.all(ws["depth"][~vis_or] == 0xFFFFFFFF)
    m = vis_or
    rec = ws["rec"]
    fields = dict(u=0, v=1, A2=2, beta=3, G2=4, opac=5)
    for k, col in fields.items():
        a = rec[m, col].view(np.uint32)
        b = pre32[k + "_f32"][m].view(np.uint32)
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, "%s differs at %d Gaussians (first %s: gpu %r oracle %r)" % (
            k, bad.size, bad[:3], rec[m, col][bad[:3]], pre32[k + "_f32"][m][bad[:3]])
    for c in range(3):
        assert np.array_equal(rec[m, 6 + c].view(np.uint32), pre32["rgb_f32"][m, c].view(np.uint32)), "rgb %d" % c
    assert np.array_equal(rec[m, 9].view(np.uint32), pre32["depth_f32"][m].view(np.uint32))
    assert np.array_equal(ws["depth"][m], pre32["depth_f32"][m].view(np.uint32))
    assert np.array_equal(ws["rect"][m], pre32["rect"][m])


def compare_lists(ws, ranges_or, list_or):
    assert ws["D"] == list_or.shape[0], (ws["D"], list_or.shape[0])
    assert np.array_equal(ws["list"].astype(np.int64), list_or.astype(np.int64))
    r = ws["ranges"].astype(np.int64)
    empty_or = ranges_or[:, 0] == ranges_or[:, 1]
    assert np.array_equal(r[~empty_or], ranges_or[~empty_or])
    assert np.all(r[empty_or, 0] == r[empty_or, 1])


def compare_image(img, al, nc_gpu, co, tol=1e-5):
    """Every pixel matches the oracle's primary result or, where a threshold
    decision was fragile, its alternative.  Returns stats."""
    img = img.astype(np.float64)
    al = al.astype(np.float64)
    e1 = np.maximum(np.abs(img - co["image"]).max(0), np.abs(al - co["alpha"]))
    e2 = np.maximum(np.abs(img - co["alt_image"]).max(0), np.abs(al - co["alt_alpha"]))
    ok1 = (e1 <= tol) & (nc_gpu == co["ncontrib"])
    ok2 = (e2 <= tol) & (nc_gpu == co["alt_ncontrib"]) & (co["fragile"] > 0)
    multi = co["fragile"] > 1
    bad = ~(ok1 | ok2) & ~multi
    return dict(max_err=float(e1[~(co["fragile"] > 0)].max()) if (~(co["fragile"] > 0)).any() else 0.0,
                n_bad=int(bad.sum()), n_fragile=int((co["fragile"] > 0).sum()), n_multi=int(multi.sum()),
                bad_idx=np.argwhere(bad)[:5])


def psnr(a, b):
    mse = float(((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2).mean())
    return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)


def oracle_stage(scene, cam, mask, planes, bg):
    """Oracle render on its single-precision decision path (tile ids / order as the GPU)."""
    pre = oracle.preprocess(scene, cam, mask, planes, "f32")
    ranges, lst = oracle.bin_tiles(pre)
    co = oracle.composite(pre, ranges, lst, bg)
    return pre, ranges, lst, co

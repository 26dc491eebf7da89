"""GPU parity of the backward (S4: compositing backward + chain rule, with the
per-Gaussian contribution) and of the prune (S5), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_16978_gb300 import contrib_prune, render
from tests.gpu_util import f64_scene, gpu_render, oracle_stage
from tests.test_gpu_render import WL

pytestmark = pytest.mark.gpu

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")
# Gradient bar: |gpu - oracle| <= GRAD_TOL * max|oracle| over each field, i.e. the
# 1e-5 absolute bar applied to each gradient field normalised by its largest
# magnitude (FP32 accumulation over the pixels of a splat against FP64).
GRAD_TOL = 1e-5


def _upstream(H, W, seed=9):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((3, H, W)).astype(np.float32), rng.standard_normal((H, W)).astype(np.float32))


def _gpu_backward(name, glm=0xFFFFFFFF):
    sc, cam, mask, planes, bg = WL[name]
    ds, rast, img, al = gpu_render(sc, cam, mask, planes, bg)
    dimg, dal = _upstream(cam.height, cam.width)
    csum = torch.zeros(sc.n, device="cuda")
    cmax = torch.zeros(sc.n, device="cuda")
    g = rast.backward(ds, cam, bg, torch.from_numpy(dimg).cuda(), torch.from_numpy(dal).cuda(), glm, csum, cmax)
    torch.cuda.synchronize()
    return sc, cam, mask, planes, bg, dimg, dal, {k: v.cpu().numpy() for k, v in g.items()}, csum.cpu().numpy(), \
        cmax.cpu().numpy()


@pytest.mark.parametrize("name", list(WL))
def test_backward_parity(name):
    sc, cam, mask, planes, bg, dimg, dal, g, csum, cmax = _gpu_backward(name)
    pre, ranges, lst, co = oracle_stage(sc, cam, mask, planes, bg)
    cb = oracle.composite_backward(pre, ranges, lst, bg, dimg, dal)
    ref = oracle.chain(f64_scene(sc), cam, pre["vis"], cb["rec_grad"])
    ok = (cb["touched_fragile"] == 0)
    stats, abs_err = {}, {}
    for f in FIELDS:
        a = g[f].reshape(sc.n, -1)[ok].astype(np.float64)
        b = ref[f].reshape(sc.n, -1)[ok]
        scale = np.abs(b).max()
        abs_err[f] = np.abs(a - b).max()
        err = abs_err[f] / scale
        stats[f] = err
        assert err <= GRAD_TOL, (f, err)
    print(name, "max gradient error, field-normalised", stats, "absolute", abs_err, "excluded", int((~ok).sum()))
    # the absolute bar with the loss taken as a mean over the pixel values
    # (dL/dimage and dL/dalpha divided by their element count)
    for f in FIELDS:
        assert abs_err[f] / (4 * cam.width * cam.height) <= 1e-5, (f, abs_err[f])
    vis = pre["vis"] > 0
    assert np.all(g["means"][~vis] == 0) and np.all(g["sh"][~vis] == 0)
    # contrib_sum is a sum of one alpha*T term per pixel at which the Gaussian
    # was blended; the 1e-5 bar applies to each term, so the sum is within
    # 1e-5 x its number of terms
    m = ok & (cb["contrib_sum"] > 0)
    err_sum = np.abs(csum[m] - cb["contrib_sum"][m])
    assert (err_sum <= 1e-5 * cb["contrib_count"][m]).all(), float((err_sum / cb["contrib_count"][m]).max())
    assert np.abs(cmax[ok] - cb["contrib_max"][ok]).max() <= 1e-5
    assert np.all(csum[~vis] == 0) and np.all(cmax[~vis] == 0)


def test_frozen_layers_get_zero_gradient():
    glm = 0b00101
    sc, cam, mask, planes, bg, dimg, dal, g, _, _ = _gpu_backward("shells_ragged", glm)
    _, _, _, _, _, _, _, gfull, _, _ = _gpu_backward("shells_ragged")
    frozen = ((glm >> sc.layer.astype(np.int64)) & 1) == 0
    for f in FIELDS:
        assert np.all(g[f][frozen] == 0)
        # float atomics sum in a run-dependent order: equal up to rounding, and
        # both runs meet the oracle bar, so they agree within it
        scale = np.abs(gfull[f]).max()
        assert np.abs(g[f][~frozen] - gfull[f][~frozen]).max() <= GRAD_TOL * scale, f


def test_autograd_function_matches_direct_backward():
    sc, cam, mask, planes, bg = WL["c1"]
    from paper_2410_16978_gb300 import DeviceScene, Rasterizer
    ds = DeviceScene.from_host(sc, requires_grad=True)
    rast = Rasterizer(sc.n, cam.width, cam.height)
    dimg, dal = _upstream(cam.height, cam.width, seed=3)
    img, al = render(ds, rast, cam, mask, planes, bg)
    loss = (img * torch.from_numpy(dimg).cuda()).sum() + (al * torch.from_numpy(dal).cuda()).sum()
    loss.backward()
    _, rast2, _, _ = gpu_render(sc, cam, mask, planes, bg)
    ds2 = DeviceScene.from_host(sc)
    g = rast2.backward(ds2, cam, bg, torch.from_numpy(dimg).cuda(), torch.from_numpy(dal).cuda())
    for f, p in zip(FIELDS, ds.params()):
        # float atomics sum in a run-dependent order: equal up to rounding
        assert (p.grad - g[f]).abs().max().item() <= GRAD_TOL * g[f].abs().max().item(), f


def test_prune_matches_oracle():
    rng = np.random.default_rng(4)
    n = 100_003
    cm = rng.uniform(0, 0.01, n).astype(np.float32)
    cm[:10] = np.float32(0.005)
    cm[10:20] = np.nextafter(np.float32(0.005), np.float32(0))
    keep, idx, nk = contrib_prune(torch.from_numpy(cm).cuda(), 0.005)
    k_or, n_or = oracle.prune(cm.astype(np.float64), float(np.float32(0.005)))
    assert int(nk.item()) == n_or
    assert np.array_equal(keep.cpu().numpy(), k_or)
    assert np.array_equal(idx.cpu().numpy()[:n_or], np.nonzero(k_or)[0])


def test_prune_edge_sizes():
    for n in (0, 1, 2047, 2048, 2049):
        cm = np.linspace(0, 0.01, max(n, 1)).astype(np.float32)[:n]
        t = torch.from_numpy(cm).cuda() if n else torch.zeros(0, device="cuda")
        keep, idx, nk = contrib_prune(t, 0.005)
        k_or, n_or = oracle.prune(cm.astype(np.float64), float(np.float32(0.005)))
        assert int(nk.item()) == n_or
        assert np.array_equal(keep.cpu().numpy(), k_or)


@pytest.mark.parametrize("glm", [0xFFFFFFFF, 0b00101])
def test_backward_overwrites_every_element(glm):
    """Gradient buffers are outputs, not accumulators: with every element NaN
    on entry, the backward leaves none (culled, frozen and live rows alike;
    a scene size that is not a multiple of the 32-row zero blocks)."""
    sc, cam, mask, planes, bg = WL["shells_ragged"]
    assert sc.n % 32 != 0
    ds, rast, img, al = gpu_render(sc, cam, mask, planes, bg)
    dimg, dal = _upstream(cam.height, cam.width)
    grads = {k: torch.full(p.shape, float("nan"), dtype=torch.float32, device="cuda")
             for k, p in zip(FIELDS, ds.params())}
    g = rast.backward(ds, cam, bg, torch.from_numpy(dimg).cuda(), torch.from_numpy(dal).cuda(), glm, grads=grads)
    torch.cuda.synchronize()
    for f in FIELDS:
        assert bool(torch.isfinite(g[f]).all()), f


def test_backward_repeats_and_follows_a_batched_render():
    """The forward writes the backward's work items (one per 256 list positions
    of every 8x8 block's longest blended prefix).  Two backward passes after
    one render, and a backward after the same view rendered inside a
    gs_render_batch launch, give the gradients of the first pass (up to the
    rounding order of the gradient atomics)."""
    from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
    sc, cam, mask, planes, bg = WL["shells_ragged"]
    ds = DeviceScene.from_host(sc)
    dimg, dal = _upstream(cam.height, cam.width)
    dI, dA = torch.from_numpy(dimg).cuda(), torch.from_numpy(dal).cuda()

    def grads(rast):
        cmax = torch.zeros(sc.n, device="cuda")
        g = rast.backward(ds, cam, bg, dI, dA, 0xFFFFFFFF, None, cmax)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in g.items()}, cmax.cpu().numpy()

    r0 = Rasterizer(sc.n, cam.width, cam.height)
    r0.render(ds, cam, mask, planes, bg)
    first, cm_first = grads(r0)
    again, cm_again = grads(r0)
    r1 = Rasterizer(sc.n, cam.width, cam.height)
    other = torch.zeros((3, cam.height, cam.width), device="cuda"), torch.zeros((cam.height, cam.width), device="cuda")
    rb = Rasterizer(sc.n, cam.width, cam.height)
    items = [dict(scene=ds.c_struct(), camera=_lib.make_camera(cam), layer_mask=mask, planes=list(planes), bg=bg,
                  workspace=r1.workspace, ws_bytes=r1.ws_bytes, image=torch.empty_like(other[0]),
                  alpha=torch.empty_like(other[1])),
             dict(scene=ds.c_struct(), camera=_lib.make_camera(cam), layer_mask=0b1, planes=[], bg=bg,
                  workspace=rb.workspace, ws_bytes=rb.ws_bytes, image=other[0], alpha=other[1])]
    _lib.gs_render_batch(items, 0)
    torch.cuda.synchronize()
    assert r1.status().error == 0
    batched, cm_batched = grads(r1)
    for k in FIELDS:
        scale = max(float(np.abs(first[k]).max()), 1e-30)
        assert np.abs(again[k] - first[k]).max() <= 1e-6 * scale, k
        assert np.abs(batched[k] - first[k]).max() <= 1e-6 * scale, k
    assert np.array_equal(cm_again, cm_first) and np.array_equal(cm_batched, cm_first)

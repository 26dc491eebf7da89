"""GPU parity of the training step (Sec. 3.2) against the FP64 oracle: the
image loss and its gradient, Adam with frozen layers, the row gather of the
prune, and one whole step (render, loss, backward, Adam) through the autograd
Functions.

Tolerances: the loss within 1e-5 relative; its gradient within 1e-5 of the
largest |dL/dX| (measured 1e-7 to 6e-7: the SSIM window moments are taken of
the values shifted by 0.5, which keeps E[x^2] - mu^2's single-precision
cancellation small for values in [0, 1]); Adam within 1e-5 of the step size."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import train as OT
from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
from paper_2410_16978_gb300.api import gather_rows
from paper_2410_16978_gb300.train import TrainConfig, Trainer, image_loss
from tests.gpu_util import f64_scene

pytestmark = pytest.mark.gpu


def _loss_inputs(rng, H, W):
    X = rng.random((3, H, W)).astype(np.float32)
    A = rng.random((H, W)).astype(np.float32)
    At = rng.random((H, W)).astype(np.float32)
    Ct = (rng.random((3, H, W)) * At[None]).astype(np.float32)
    return X, A, Ct, At


@pytest.mark.parametrize("H,W,lam,w_a", [(37, 53, 0.2, 0.8), (128, 96, 0.2, 0.0), (9, 300, 1.0, 0.3), (1, 1, 0.2, 1.0)])
def test_image_loss_matches_oracle(H, W, lam, w_a):
    rng = np.random.default_rng(H * 1000 + W)
    X, A, Ct, At = _loss_inputs(rng, H, W)
    bg = (0.3, 0.6, 0.1)
    L, dX, dA = OT.loss_grad(X, A, Ct, At, bg, lam, w_a)
    t = [torch.from_numpy(a).cuda() for a in (X, A, Ct, At)]
    ws = torch.empty(_lib.gs_image_loss_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    loss = torch.empty((), device="cuda")
    gX = torch.empty_like(t[0])
    gA = torch.empty_like(t[1])
    _lib.gs_image_loss(t[0], t[1] if w_a else None, t[2], t[3], bg, W, H, lam, w_a, ws, ws.numel(), loss, gX, gA, 0)
    torch.cuda.synchronize()
    assert abs(float(loss) - L) <= 1e-5 * abs(L)
    e = np.abs(gX.cpu().numpy() - dX).max() / np.abs(dX).max()
    print("loss gradient error (of max |dL/dX|):", e)
    assert e <= 1e-5, e
    if w_a:
        assert np.abs(gA.cpu().numpy() - dA).max() <= 1e-6 * np.abs(dA).max()
    else:
        assert float(gA.abs().max()) == 0.0


def test_image_loss_autograd_and_identity():
    rng = np.random.default_rng(9)
    X, A, Ct, At = _loss_inputs(rng, 40, 24)
    bg = (0.5, 0.5, 0.5)
    Y = OT.target_under(bg, Ct, At).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (X, A, Ct, At)]
    x = t[0].clone().requires_grad_(True)
    a = t[1].clone().requires_grad_(True)
    loss = image_loss(x, a, t[2], t[3], bg, 0.2, 0.8)
    loss.backward()
    _, dX, dA = OT.loss_grad(X, A, Ct, At, bg, 0.2, 0.8)
    assert np.abs(x.grad.cpu().numpy() - dX).max() <= 1e-5 * np.abs(dX).max()
    assert np.abs(a.grad.cpu().numpy() - dA).max() <= 1e-6 * np.abs(dA).max()
    # image equal to the target (and alpha to its alpha): SSIM 1, loss 0
    z = image_loss(torch.from_numpy(Y).cuda(), t[3], t[2], t[3], bg, 0.2, 0.8)
    assert abs(float(z)) < 1e-6


@pytest.mark.parametrize("mask,unaligned", [(0b110, False), (0xFFFFFFFF, False), (0b110, True)])
def test_adam_matches_oracle_with_frozen_layers(mask, unaligned):
    """Adam against the oracle: layer 0 frozen (or every layer trainable),
    arrays whose lengths are not multiples of four, and moments 4 bytes off a
    16-byte boundary (the element-wise path instead of the 16-byte one)."""
    rng = np.random.default_rng(3)
    n, K = 301, 16
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]
    p0 = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    layer = rng.integers(0, 3, n).astype(np.uint8)
    lr = (1e-3, 5e-3, 2e-3, 5e-2, 2.5e-3)
    P = [torch.from_numpy(a.copy()).cuda() for a in p0]
    if unaligned:
        M = [torch.zeros(a.numel() + 1, device="cuda")[1:].view(a.shape) for a in P]
        V = [torch.zeros(a.numel() + 1, device="cuda")[1:].view(a.shape) for a in P]
    else:
        M = [torch.zeros_like(a) for a in P]
        V = [torch.zeros_like(a) for a in P]
    frozen = ((mask >> layer.astype(np.int64)) & 1) == 0
    sc = DeviceScene(*P, torch.from_numpy(layer).cuda(), 3)
    ref = [(a.astype(np.float64), np.zeros(a.shape), np.zeros(a.shape)) for a in p0]
    for t in range(1, 4):
        gr = [rng.standard_normal(s).astype(np.float32) for s in shapes]
        G = [torch.from_numpy(a).cuda() for a in gr]
        g = _lib.gs_grads()
        g.means, g.log_scales, g.quats, g.opacity_logit, g.sh = (x.data_ptr() for x in G)
        st = _lib.gs_adam_state()
        for k in range(5):
            st.m[k], st.v[k] = M[k].data_ptr(), V[k].data_ptr()
        _lib.gs_adam_step(sc.c_struct(), g, st, lr, 0.9, 0.999, 1e-15, t, mask, 0)
        ref = [OT.adam_step(r[0], gr[k], r[1], r[2], t, lr[k], frozen_rows=frozen)
               for k, r in enumerate(ref)]
    torch.cuda.synchronize()
    for k in range(5):
        got = P[k].cpu().numpy()
        assert np.array_equal(got[frozen], p0[k][frozen])                  # frozen: untouched
        assert np.abs(got - ref[k][0]).max() <= 1e-5 * lr[k] * 3 + 4e-7 * np.abs(ref[k][0]).max(), k
        assert np.allclose(M[k].cpu().numpy(), ref[k][1], rtol=1e-5, atol=1e-6)
        assert np.allclose(V[k].cpu().numpy(), ref[k][2], rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("dtype,shape", [(torch.float32, (3,)), (torch.float16, (3,)), (torch.uint8, ()),
                                         (torch.float32, (16, 3)), (torch.bfloat16, (4,))])
def test_gather_rows(dtype, shape):
    rng = np.random.default_rng(1)
    n = 1000
    src = torch.from_numpy(rng.integers(0, 200, (n,) + shape).astype(np.float32)).to(dtype).cuda()
    keep = np.sort(rng.choice(n, 357, replace=False)).astype(np.int32)
    got = gather_rows(src, torch.from_numpy(keep).cuda())
    torch.cuda.synchronize()
    assert torch.equal(got.cpu(), src.cpu()[torch.from_numpy(keep).long()])


def _small_training_case():
    rng = np.random.default_rng(21)
    sc = synth.shell_scene(rng, [900, 700], (0.8, 0.45), sh_degree=1)
    cams = synth.fibonacci_cameras(2, radius=3.2, width=72, height=56)
    return sc, cams


def test_training_step_gradients_match_oracle():
    """One step through RenderFunction + ImageLossFunction: the gradients
    reaching Adam equal the oracle's (render from the same single-precision
    projection, FP64 compositing, loss gradient, backward and chain rule)
    within 1e-5 of each field's largest magnitude; frozen layers get zero
    gradient and keep their parameters.  Gaussians touched by a fragile
    threshold decision, or blended at a pixel where 0 < |X - Y| < 1e-4 (the
    sign of the L1 term is not decided by the arithmetic there), are not
    compared."""
    sc, cams = _small_training_case()
    cam = cams[0]
    rng = np.random.default_rng(5)
    tgt = oracle.render(sc.copy(), cam, 0xFFFFFFFF, (), (0.0, 0.0, 0.0))
    Ct = tgt["image"].astype(np.float32)                    # rendered on black: premultiplied colour
    At = tgt["alpha"].astype(np.float32)
    sc2 = sc.copy()
    sc2.means = (sc2.means + rng.normal(0, 0.01, sc2.means.shape)).astype(np.float32)
    sc2.sh = (sc2.sh + rng.normal(0, 0.05, sc2.sh.shape)).astype(np.float32)
    bg = tuple(float(v) for v in rng.uniform(0, 1, 3))
    mask = 0b10                                             # train layer 1, layer 0 frozen
    ds = DeviceScene.from_host(sc2)
    p_before = [p.detach().clone() for p in ds.params()]
    tr = Trainer(ds, [cam], TrainConfig(train_layer_mask=mask, w_alpha=0.8))
    fw = oracle.render(sc2, cam, 0xFFFFFFFF, (), bg, precision="f32")
    _, dX, dA = OT.loss_grad(fw["image"], fw["alpha"], Ct, At, bg, 0.2, 0.8)
    ref = oracle.render_backward(f64_scene(sc2), cam, fw, bg, dX, dA, grad_layer_mask=mask)
    tr.step(0, torch.from_numpy(Ct).cuda(), torch.from_numpy(At).cuda(), bg)
    torch.cuda.synchronize()
    # tiles with an undecided L1 sign
    Y = OT.target_under(bg, Ct, At)
    d_rgb, d_a = np.abs(fw["image"] - Y), np.abs(fw["alpha"] - At)
    # exact zeros (background on both sides) are decided; tiny non-zero gaps are not
    close = ((d_rgb > 0) & (d_rgb < 1e-4)).any(0) | ((d_a > 0) & (d_a < 1e-4))
    # Gaussians blended at such a pixel: non-zero colour gradient for dL/dC = 1 there
    ind = np.repeat(close[None].astype(np.float64), 3, 0)
    hit = oracle.composite_backward(fw["pre"], fw["ranges"], fw["list"], bg, ind)["rec_grad"][:, 6] != 0
    keep = (ref["touched_fragile"] == 0) & ~hit & (fw["pre"]["vis"] > 0)
    assert keep.sum() >= 100, keep.sum()
    frozen = sc2.layer == 0
    for k, f in enumerate(("means", "log_scales", "quats", "opacity_logit", "sh")):
        gg = tr.scene.params()[k].grad.cpu().numpy().reshape(sc2.n, -1).astype(np.float64)
        rr = ref[f].reshape(sc2.n, -1)
        assert np.all(gg[frozen] == 0.0), f
        err = np.abs(gg[keep] - rr[keep]).max() / max(np.abs(rr[keep]).max(), 1e-30)
        assert err <= 1e-5, (f, err)
        after = tr.scene.params()[k].detach().cpu().numpy().reshape(sc2.n, -1)
        assert np.array_equal(after[frozen], p_before[k].cpu().numpy().reshape(sc2.n, -1)[frozen]), f
    assert tr.t == 1


def test_training_prune_compacts_parameters_and_moments():
    sc, cams = _small_training_case()
    ds = DeviceScene.from_host(sc)
    tr = Trainer(ds, cams, TrainConfig(prune_threshold=0.05))
    rng = np.random.default_rng(2)
    for v in range(2):
        tgt_rgb = torch.from_numpy(rng.random((3, 56, 72)).astype(np.float32) * 0.5).cuda()
        tgt_a = torch.full((56, 72), 0.5, device="cuda")
        tr.step(v, tgt_rgb, tgt_a, (0.2, 0.2, 0.2))
    cm = tr.contrib_max.cpu().numpy()
    params = [p.detach().cpu().numpy() for p in tr.scene.params()]
    moments = [m.cpu().numpy() for m in tr.m]
    keep_ref, n_ref = oracle.prune(cm, 0.05)
    n = tr.prune()
    torch.cuda.synchronize()
    assert n == n_ref == int(keep_ref.sum()) and 0 < n < sc.n
    for a, b in zip(tr.scene.params(), params):
        assert np.array_equal(a.detach().cpu().numpy(), b[keep_ref.astype(bool)])
    for a, b in zip(tr.m, moments):
        assert np.array_equal(a.cpu().numpy(), b[keep_ref.astype(bool)])
    assert tr.scene.n == n and tr.contrib_max.shape[0] == n


def test_activity_accumulate_and_prune_match_oracle():
    """Activity of three Adam steps (frozen layer 0) against the oracle's norms
    of its own updates; the prune decision bit-exact on the GPU's activity."""
    rng = np.random.default_rng(8)
    n, K = 257, 16
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]
    p0 = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    layer = rng.integers(0, 3, n).astype(np.uint8)
    mask = 0b110
    lr = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)
    P = [torch.from_numpy(a.copy()).cuda() for a in p0]
    M = [torch.zeros_like(a) for a in P]
    V = [torch.zeros_like(a) for a in P]
    L = torch.from_numpy(layer).cuda()
    sc = DeviceScene(*P, L, 3)
    act = torch.zeros(n, device="cuda")
    ref = [(a.astype(np.float64), np.zeros(a.shape), np.zeros(a.shape)) for a in p0]
    ref_act = np.zeros(n)
    frozen = ((mask >> layer.astype(np.int64)) & 1) == 0
    for t in range(1, 4):
        gr = [rng.standard_normal(s).astype(np.float32) for s in shapes]
        G = [torch.from_numpy(a).cuda() for a in gr]
        g = _lib.gs_grads()
        g.means, g.log_scales, g.quats, g.opacity_logit, g.sh = (x.data_ptr() for x in G)
        st = _lib.gs_adam_state()
        for k in range(5):
            st.m[k], st.v[k] = M[k].data_ptr(), V[k].data_ptr()
        _lib.gs_adam_step(sc.c_struct(), g, st, lr, 0.9, 0.999, 1e-15, t, mask, 0)
        _lib.gs_activity_accumulate(st, L, n, 3, lr, 0.9, 0.999, 1e-15, t, mask, act, 0)
        new = [OT.adam_step(r[0], gr[k], r[1], r[2], t, lr[k], frozen_rows=frozen) for k, r in enumerate(ref)]
        d = [new[k][0] - ref[k][0] for k in range(5)]
        ref_act += OT.activity_sample(d[0], d[4], d[1])
        ref = new
    torch.cuda.synchronize()
    a = act.cpu().numpy().astype(np.float64)
    assert np.all(a[frozen] == 0.0)
    assert np.abs(a - ref_act).max() <= 1e-5 * np.abs(ref_act).max()
    # decision on the GPU's own activity (two samples: act * 0.5 is exact in
    # both precisions), threshold inside its range
    thr = float(np.float32(np.median(a[~frozen]) / 2.0))
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    nk = torch.empty(1, dtype=torch.int64, device="cuda")
    wsb = _lib.gs_prune_workspace_size(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    _lib.gs_activity_prune(act, L, n, mask, 2.0, thr, keep, idx, nk, ws, wsb, 0)
    torch.cuda.synchronize()
    want = OT.activity_prune(a, 2, thr, ~frozen)
    got = keep.cpu().numpy().astype(bool)
    assert np.array_equal(got, want)
    k = int(nk.item())
    assert k == int(want.sum()) and np.array_equal(idx.cpu().numpy()[:k], np.nonzero(want)[0])


def test_trainer_activity_prune_keeps_frozen_layers():
    sc, cams = _small_training_case()
    ds = DeviceScene.from_host(sc)
    cfg = TrainConfig(train_layer_mask=0b10, activity_prune=True, activity_interval=3, activity_threshold=1e9)
    tr = Trainer(ds, cams, cfg)
    rng = np.random.default_rng(4)
    n_frozen = int((sc.layer == 0).sum())
    for v in range(3):
        tr.step(v % 2, torch.from_numpy(rng.random((3, 56, 72)).astype(np.float32) * 0.5).cuda(),
                torch.full((56, 72), 0.5, device="cuda"), (0.3, 0.3, 0.3))
    torch.cuda.synchronize()
    # a huge threshold removes every trainable Gaussian and no frozen one
    assert tr.scene.n == n_frozen and tr.activity_removed == sc.n - n_frozen
    assert np.all(tr.scene.layer.cpu().numpy() == 0)
    assert tr.activity_samples == 0 and abs(tr.activity_threshold - 1e9 * 0.975) < 1e3
    assert tr.m[0].shape[0] == n_frozen and tr.contrib_max.shape[0] == n_frozen

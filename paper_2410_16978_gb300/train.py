"""Training step of the layered model (Sec. 3.2): render through the
autograd Function, image loss with the alpha channel against a target under a
random background, backward with per-Gaussian contributions, Adam on the
trainable layers, contribution pruning, and the activity-based inactive
pruning of Sec. 3.2.2.

Every step runs in libgs.so kernels (gs_render, gs_image_loss,
gs_render_backward, gs_adam_step, gs_activity_accumulate, gs_activity_prune,
gs_contrib_prune, gs_gather_rows); PyTorch holds the tensors and chains the
two autograd Functions.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import torch

from . import _lib
from .api import DeviceScene, Rasterizer, _require_cuda, _stream_handle, contrib_prune, gather_rows, render

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")


class ImageLossFunction(torch.autograd.Function):
    """loss = (1 - lam) L1 + lam (1 - SSIM) + w_alpha L1(alpha) via gs_image_loss;
    the gradient comes from the same launch and is scaled by the upstream one."""

    @staticmethod
    def forward(ctx, image, alpha, target_rgb, target_alpha, bg, lam: float, w_alpha: float, workspace):
        H, W = int(image.shape[1]), int(image.shape[2])
        loss = torch.empty((), dtype=torch.float32, device=image.device)
        d_img = torch.empty_like(image)
        d_al = torch.empty_like(alpha) if alpha is not None else None
        ws = workspace if workspace is not None else torch.empty(_lib.gs_image_loss_workspace_size(W, H),
                                                                 dtype=torch.uint8, device=image.device)
        _lib.gs_image_loss(image, alpha if w_alpha else None, target_rgb, target_alpha, bg, W, H, lam, w_alpha, ws,
                           ws.numel(), loss, d_img, d_al, _stream_handle(None))
        ctx.save_for_backward(d_img, d_al if d_al is not None else torch.empty(0, device=image.device))
        ctx.has_alpha = d_al is not None
        return loss

    @staticmethod
    def backward(ctx, g):
        d_img, d_al = ctx.saved_tensors
        # g is the scalar upstream gradient (1 for loss.backward()); scaling is plumbing
        return (d_img * g, (d_al * g) if ctx.has_alpha else None, None, None, None, None, None, None)


def image_loss(image, alpha, target_rgb, target_alpha, bg, lam=0.2, w_alpha=0.0, workspace=None):
    return ImageLossFunction.apply(image, alpha, target_rgb, target_alpha, tuple(float(v) for v in bg), float(lam),
                                   float(w_alpha), workspace)


@dataclasses.dataclass
class TrainConfig:
    lr: Sequence[float] = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)   # means, log-scales, quats, opacity, SH
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    lam: float = 0.2                     # D-SSIM weight
    w_alpha: float = 0.8                 # alpha L1 weight
    train_layer_mask: int = 0xFFFFFFFF   # layers being optimised (the rest are frozen)
    prune_threshold: float = 0.005
    activity_prune: bool = False         # inactive pruning of Sec. 3.2.2
    activity_interval: int = 100         # dR: steps per activity average
    activity_threshold: float = 0.015    # T0
    activity_decay: float = 0.975


class Trainer:
    """Optimises a float32 DeviceScene against per-view targets.  One step =
    one view: forward, loss, backward (gradients of the trainable layers and
    the blend weights of every Gaussian), Adam.  ``prune()`` removes the
    Gaussians whose largest blend weight since the last prune is below the
    threshold, with their Adam moments.  With ``activity_prune`` every step
    also accumulates each trainable Gaussian's activity, and every
    ``activity_interval`` steps the inactive ones are removed."""

    def __init__(self, scene: DeviceScene, cameras: Sequence, config: TrainConfig = TrainConfig(),
                 dup_capacity: Optional[int] = None):
        if scene.sh_dtype != "f32" or scene.sr_dtype != "f32":
            raise ValueError("training needs float32 parameters")
        self.cfg = config
        self.cameras = list(cameras)
        self.scene = scene
        for p in scene.params():
            p.requires_grad_(True)
        self.device = scene.means.device
        self.m = [torch.zeros_like(p, dtype=torch.float32) for p in scene.params()]
        self.v = [torch.zeros_like(p, dtype=torch.float32) for p in scene.params()]
        self.t = 0
        self.dup_capacity = dup_capacity
        self._rasts = {}
        self._loss_ws = {}
        self.contrib_max = torch.zeros(scene.n, device=self.device)
        self.contrib_sum = torch.zeros(scene.n, device=self.device)
        self.activity = torch.zeros(scene.n, device=self.device)
        self.activity_samples = 0
        self.activity_threshold = float(config.activity_threshold)
        self.activity_removed = 0

    def _rast(self, cam) -> Rasterizer:
        key = (int(cam.width), int(cam.height))
        r = self._rasts.get(key)
        if r is None or r.n != self.scene.n:
            r = Rasterizer(self.scene.n, cam.width, cam.height, device=self.device, dup_capacity=self.dup_capacity)
            self._rasts[key] = r
        return r

    def _lws(self, W, H):
        key = (W, H)
        if key not in self._loss_ws:
            self._loss_ws[key] = torch.empty(_lib.gs_image_loss_workspace_size(W, H), dtype=torch.uint8,
                                             device=self.device)
        return self._loss_ws[key]

    def step(self, view: int, target_rgb: torch.Tensor, target_alpha: torch.Tensor, bg=(0.0, 0.0, 0.0),
             layer_mask: int = 0xFFFFFFFF, planes=()):
        """One optimisation step on camera ``view``; returns the loss (device scalar)."""
        for t, nm in ((target_rgb, "target_rgb"), (target_alpha, "target_alpha")):
            _require_cuda(t, nm)
        cam = self.cameras[view]
        sc = self.scene
        for p in sc.params():
            p.grad = None
        img, al = render(sc, self._rast(cam), cam, layer_mask, planes, bg, self.cfg.train_layer_mask,
                         self.contrib_sum, self.contrib_max)
        loss = image_loss(img, al, target_rgb, target_alpha, bg, self.cfg.lam, self.cfg.w_alpha,
                          self._lws(cam.width, cam.height))
        loss.backward()
        self.t += 1
        with torch.no_grad():
            g = _lib.gs_grads()
            grads = [p.grad for p in sc.params()]
            g.means, g.log_scales, g.quats, g.opacity_logit, g.sh = (x.data_ptr() for x in grads)
            st = _lib.gs_adam_state()
            for k in range(5):
                st.m[k] = self.m[k].data_ptr()
                st.v[k] = self.v[k].data_ptr()
            _lib.gs_adam_step(sc.c_struct(), g, st, self.cfg.lr, self.cfg.beta1, self.cfg.beta2, self.cfg.eps, self.t,
                              self.cfg.train_layer_mask, _stream_handle(None))
            if self.cfg.activity_prune:
                _lib.gs_activity_accumulate(st, sc.layer, sc.n, sc.sh_degree, self.cfg.lr, self.cfg.beta1,
                                            self.cfg.beta2, self.cfg.eps, self.t, self.cfg.train_layer_mask,
                                            self.activity, _stream_handle(None))
                self.activity_samples += 1
        if self.cfg.activity_prune and self.activity_samples == self.cfg.activity_interval:
            self.activity_prune()
        return loss.detach()

    def _apply_keep(self, keep_index, n: int):
        idx = keep_index[:n]
        with torch.no_grad():
            sub = self.scene.subset(idx)
            self.m = [gather_rows(a, idx) for a in self.m]
            self.v = [gather_rows(a, idx) for a in self.v]
            self.contrib_max = gather_rows(self.contrib_max, idx)
            self.contrib_sum = gather_rows(self.contrib_sum, idx)
            self.activity = gather_rows(self.activity, idx)
        self.scene = sub
        for p in sub.params():
            p.requires_grad_(True)

    def activity_prune(self) -> int:
        """Inactive pruning (Sec. 3.2.2): removes the trainable Gaussians whose
        average activity over the samples since the last decision is at or
        below the threshold, then decays the threshold and restarts the
        average.  Returns the number kept."""
        sc = self.scene
        keep = torch.empty(sc.n, dtype=torch.uint8, device=self.device)
        keep_index = torch.empty(sc.n, dtype=torch.int32, device=self.device)
        n_keep = torch.empty(1, dtype=torch.int64, device=self.device)
        wsb = _lib.gs_prune_workspace_size(sc.n)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=self.device)
        _lib.gs_activity_prune(self.activity, sc.layer, sc.n, self.cfg.train_layer_mask, self.activity_samples,
                               self.activity_threshold, keep, keep_index, n_keep, ws, wsb, _stream_handle(None))
        n = int(n_keep.item())
        self.activity_removed += sc.n - n
        if n < sc.n:
            self._apply_keep(keep_index, n)
        self.activity.zero_()
        self.activity_samples = 0
        self.activity_threshold *= self.cfg.activity_decay
        return n

    def prune(self) -> int:
        """Applies the contribution prune; returns the number of Gaussians kept."""
        keep, keep_index, n_keep = contrib_prune(self.contrib_max, self.cfg.prune_threshold)
        n = int(n_keep.item())
        self._apply_keep(keep_index, n)
        self.contrib_max.zero_()
        self.contrib_sum.zero_()
        return n

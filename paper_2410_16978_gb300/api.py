"""PyTorch-facing layer over the C ABI: device scene tensors, workspace
ownership, the contribution prune and the autograd Function.

PyTorch provides device memory, streams and autograd plumbing only; every step
of the render and its backward runs in the CUDA kernels of libgs.so.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import torch

from . import _lib

_DT = {"f32": (_lib.GS_DTYPE_F32, torch.float32), "f16": (_lib.GS_DTYPE_F16, torch.float16),
       "bf16": (_lib.GS_DTYPE_BF16, torch.bfloat16), "cb": (_lib.GS_DTYPE_SH_CODEBOOK, torch.float32)}


def _require_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class DeviceScene:
    """Layered Gaussian scene resident in device memory (structure of arrays).

    ``sh_dtype`` / ``sr_dtype`` select the storage of the SH coefficients and
    of the log-scales + quaternions: ``"f32"``, ``"f16"`` or ``"bf16"``.
    """

    def __init__(self, means, log_scales, quats, opacity_logit, sh, layer, sh_degree: int,
                 sh_dtype: str = "f32", sr_dtype: str = "f32", sh_index=None, sh_table=None):
        self.means = means
        self.log_scales = log_scales
        self.quats = quats
        self.opacity_logit = opacity_logit
        self.sh = sh
        self.layer = layer
        self.sh_degree = int(sh_degree)
        self.sh_dtype = sh_dtype
        self.sr_dtype = sr_dtype
        self.sh_index = sh_index      # codebook storage ("cb"): uint16 [N]
        self.sh_table = sh_table      # codebook storage: float16 [rows][R]
        names = ["means", "log_scales", "quats", "opacity_logit", "sh", "layer"]
        if sh_dtype == "cb":
            if sh_index is None or sh_table is None:
                raise ValueError("codebook storage needs sh_index and sh_table")
            names += ["sh_index", "sh_table"]
        for name in names:
            _require_cuda(getattr(self, name), name)

    @classmethod
    def from_host(cls, scene, device="cuda", sh_dtype="f32", sr_dtype="f32", requires_grad=False):
        """From a synth.Scene (numpy arrays)."""
        def t(a, dt):
            return torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        shdt, srdt = _DT[sh_dtype][1], _DT[sr_dtype][1]
        obj = cls(t(scene.means, torch.float32), t(scene.log_scales, srdt), t(scene.quats, srdt),
                  t(scene.opacity_logit, torch.float32), t(scene.sh, shdt),
                  torch.as_tensor(scene.layer).to(device=device, dtype=torch.uint8).contiguous(),
                  scene.sh_degree, sh_dtype, sr_dtype)
        if requires_grad:
            for p in obj.params():
                p.requires_grad_(True)
        return obj

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def params(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logit, self.sh]

    def c_struct(self, means=None, log_scales=None, quats=None, opacity_logit=None, sh=None) -> _lib.gs_scene:
        s = _lib.gs_scene()
        s.means = (means if means is not None else self.means).data_ptr()
        s.log_scales = (log_scales if log_scales is not None else self.log_scales).data_ptr()
        s.quats = (quats if quats is not None else self.quats).data_ptr()
        s.opacity_logit = (opacity_logit if opacity_logit is not None else self.opacity_logit).data_ptr()
        s.sh = (sh if sh is not None else self.sh).data_ptr()
        s.layer = self.layer.data_ptr()
        s.n = self.n
        s.sh_degree = self.sh_degree
        s.dtype_sh = _DT[self.sh_dtype][0]
        s.dtype_scale_rot = _DT[self.sr_dtype][0]
        if self.sh_dtype == "cb":
            s.sh_index = self.sh_index.data_ptr()
            s.sh_table = self.sh_table.data_ptr()
            s.sh_table_rows = int(self.sh_table.shape[0])
        return s

    def subset(self, keep_index: torch.Tensor, stream=None) -> "DeviceScene":
        """The Gaussians keep_index (device int32, in order), gathered by gs_gather_rows."""
        return DeviceScene(*(gather_rows(a, keep_index, stream) for a in self.params()),
                           gather_rows(self.layer, keep_index, stream), self.sh_degree, self.sh_dtype,
                           self.sr_dtype)


def gather_rows(src: torch.Tensor, keep_index: torch.Tensor, stream=None) -> torch.Tensor:
    """dst[i] = src[keep_index[i]] along the first axis (gs_gather_rows)."""
    _require_cuda(src, "src")
    _require_cuda(keep_index, "keep_index")
    if keep_index.dtype != torch.int32:
        raise ValueError("keep_index must be int32")
    n = int(keep_index.shape[0])
    row_bytes = max(1, int(math.prod(src.shape[1:]))) * src.element_size()
    dst = torch.empty((n,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    if n:
        _lib.gs_gather_rows(src, dst, row_bytes, keep_index, n, _stream_handle(stream))
    return dst


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Rasterizer:
    """Owns one render workspace (device memory for the binning lists and the
    forward state that the backward reads).  One Rasterizer per in-flight view.

    ``dup_capacity`` is the number of (tile, Gaussian) pairs the workspace can
    hold; by default 8 per Gaussian.  With ``check=True`` a render reads the
    device status word (a stream synchronisation) and, when the frame needed
    more pairs, grows the workspace and renders again."""

    def __init__(self, n: int, width: int, height: int, device="cuda", dup_capacity: Optional[int] = None):
        self.n, self.width, self.height = int(n), int(width), int(height)
        self.device = torch.device(device)
        cap = int(dup_capacity) if dup_capacity is not None else max(1 << 16, 8 * self.n)
        self._alloc(cap)

    def _alloc(self, cap: int):
        self.dup_capacity = int(cap)
        self.ws_bytes = _lib.gs_render_workspace_size(self.n, self.width, self.height, self.dup_capacity)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def status(self, stream=None) -> _lib.gs_status:
        return _lib.gs_read_status(self.workspace, _stream_handle(stream))

    def render(self, scene: DeviceScene, camera, layer_mask: int = 0xFFFFFFFF, planes: Sequence = (),
               bg=(0.0, 0.0, 0.0), image: Optional[torch.Tensor] = None, alpha: Optional[torch.Tensor] = None,
               stream=None, check: bool = True, _c_scene=None):
        if scene.n != self.n:
            raise ValueError("scene has %d Gaussians, rasterizer was sized for %d" % (scene.n, self.n))
        cam = camera if isinstance(camera, _lib.gs_camera) else _lib.make_camera(camera)
        if (cam.width, cam.height) != (self.width, self.height):
            raise ValueError("camera size differs from the rasterizer's")
        H, W = self.height, self.width
        if image is None:
            image = torch.empty((3, H, W), dtype=torch.float32, device=self.device)
        if alpha is None:
            alpha = torch.empty((H, W), dtype=torch.float32, device=self.device)
        cs = _c_scene if _c_scene is not None else scene.c_struct()
        sh = _stream_handle(stream)
        attempts = 4
        for attempt in range(attempts):
            _lib.gs_render(cs, cam, layer_mask, list(planes), bg, self.workspace, self.ws_bytes, image, alpha, sh)
            if not check:
                break
            st = _lib.gs_read_status(self.workspace, sh)
            if st.error == _lib.GS_OK:
                break
            if st.error != _lib.GS_ERR_WORKSPACE:
                raise _lib.GsError(st.error, "device status")
            if attempt + 1 == attempts:
                # The workspace of the failed render stays, so its status word
                # still describes that render.
                raise _lib.GsError(_lib.GS_ERR_WORKSPACE,
                                   "pair list still overflows after %d regrowths" % (attempts - 1))
            self._alloc(int(math.ceil(st.n_dup * 1.25)) + 1024)
        return image, alpha

    def backward(self, scene: DeviceScene, camera, bg, dL_dimage=None, dL_dalpha=None,
                 grad_layer_mask: int = 0xFFFFFFFF, contrib_sum=None, contrib_max=None, grads=None, stream=None,
                 _c_scene=None):
        cam = camera if isinstance(camera, _lib.gs_camera) else _lib.make_camera(camera)
        if grads is None:
            grads = {k: torch.empty(p.shape, dtype=torch.float32, device=self.device)
                     for k, p in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), scene.params())}
        g = _lib.gs_grads()
        g.means = grads["means"].data_ptr()
        g.log_scales = grads["log_scales"].data_ptr()
        g.quats = grads["quats"].data_ptr()
        g.opacity_logit = grads["opacity_logit"].data_ptr()
        g.sh = grads["sh"].data_ptr()
        for t, nm in ((dL_dimage, "dL_dimage"), (dL_dalpha, "dL_dalpha")):
            if t is not None:
                _require_cuda(t, nm)
        cs = _c_scene if _c_scene is not None else scene.c_struct()
        _lib.gs_render_backward(cs, cam, bg, self.workspace, self.ws_bytes, dL_dimage, dL_dalpha, grad_layer_mask,
                                g, contrib_sum, contrib_max, _stream_handle(stream))
        return grads


def contrib_prune(contrib_max: torch.Tensor, threshold: float = 0.005, stream=None, workspace=None):
    """keep = contrib_max >= threshold.  Returns (keep uint8 [N], keep_index int32 [N]
    whose first n_keep entries are the kept indices, n_keep int64 device scalar)."""
    _require_cuda(contrib_max, "contrib_max")
    n = int(contrib_max.shape[0])
    dev = contrib_max.device
    keep = torch.empty(n, dtype=torch.uint8, device=dev)
    keep_index = torch.empty(n, dtype=torch.int32, device=dev)
    n_keep = torch.empty(1, dtype=torch.int64, device=dev)
    wsb = _lib.gs_prune_workspace_size(n)
    if workspace is None:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
    _lib.gs_contrib_prune(contrib_max, n, threshold, keep, keep_index, n_keep, workspace, wsb,
                          _stream_handle(stream))
    return keep, keep_index, n_keep


class RenderFunction(torch.autograd.Function):
    """image, alpha = render(means, log_scales, quats, opacity_logit, sh); the
    backward runs gs_render_backward and also accumulates the per-Gaussian
    blend weights into ``contrib_sum`` / ``contrib_max`` when given."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, scene: DeviceScene, rast: Rasterizer, camera,
                layer_mask: int, planes, bg, grad_layer_mask: int, contrib_sum, contrib_max):
        cs = scene.c_struct(means, log_scales, quats, opacity_logit, sh)
        image, alpha = rast.render(scene, camera, layer_mask, planes, bg, _c_scene=cs)
        ctx.save_for_backward(means, log_scales, quats, opacity_logit, sh)
        ctx.meta = (scene, rast, camera, bg, grad_layer_mask, contrib_sum, contrib_max)
        return image, alpha

    @staticmethod
    def backward(ctx, d_image, d_alpha):
        means, log_scales, quats, opacity_logit, sh = ctx.saved_tensors
        scene, rast, camera, bg, glm, csum, cmax = ctx.meta
        cs = scene.c_struct(means, log_scales, quats, opacity_logit, sh)
        d_image = d_image.contiguous() if d_image is not None else None
        d_alpha = d_alpha.contiguous() if d_alpha is not None else None
        g = rast.backward(scene, camera, bg, d_image, d_alpha, glm, csum, cmax, _c_scene=cs)
        outs = [g["means"], g["log_scales"].to(log_scales.dtype), g["quats"].to(quats.dtype), g["opacity_logit"],
                g["sh"].to(sh.dtype)]
        return (*outs, None, None, None, None, None, None, None, None, None)


def render(scene: DeviceScene, rast: Rasterizer, camera, layer_mask=0xFFFFFFFF, planes=(), bg=(0.0, 0.0, 0.0),
           grad_layer_mask=0xFFFFFFFF, contrib_sum=None, contrib_max=None):
    """Differentiable render of ``scene`` (its parameter tensors may require grad)."""
    return RenderFunction.apply(scene.means, scene.log_scales, scene.quats, scene.opacity_logit, scene.sh, scene,
                                rast, camera, layer_mask, tuple(planes), tuple(float(v) for v in bg),
                                grad_layer_mask, contrib_sum, contrib_max)

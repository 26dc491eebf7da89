"""Seeded synthetic layered Gaussian scenes and cameras.

The paper's CT datasets and trained models are not available, so every
workload is synthetic and shaped like the paper's scenes (Sec. 4.2 and
Table 1: nested anatomical layers of 10^5..10^6 Gaussians, stereo VR frames,
transparent backgrounds).  Everything here is plain random-number drawing and
camera-pose construction; nothing in this file evaluates the rendering method.

Conventions
-----------
* ``means`` float32 [N,3]; ``log_scales`` float32 [N,3]; ``quats`` float32
  [N,4] in (w, x, y, z) order; ``opacity_logit`` float32 [N]; ``sh`` float32
  [N, K, 3] with K = (deg+1)^2 coefficients per colour channel; ``layer``
  uint8 [N] with values in [0, 31].
* Cameras are world-to-camera (p = R mu + t) with OpenCV axes (x right, y down,
  z forward), principal point at the image centre.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

BASE_SEED = 2410169780


def config_seed(index: int) -> int:
    """Seed of workload ``index`` (1-based)."""
    return BASE_SEED + int(index)


@dataclasses.dataclass
class Camera:
    R: np.ndarray            # float32 [3,3], world -> camera rotation (row-major)
    t: np.ndarray            # float32 [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2

    def copy(self) -> "Camera":
        return dataclasses.replace(self, R=self.R.copy(), t=self.t.copy())


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    layer: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx], self.log_scales[idx], self.quats[idx],
                     self.opacity_logit[idx], self.sh[idx], self.layer[idx],
                     self.sh_degree)

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                     self.opacity_logit.copy(), self.sh.copy(), self.layer.copy(),
                     self.sh_degree)


def _normalize(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v)


def look_at_camera(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_x_deg=50.0,
                   width=128, height=128, znear=0.2) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target`` (OpenCV axes, square pixels)."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    z = _normalize(target - eye)
    if abs(float(np.dot(z, _normalize(up)))) > 0.999:
        up = np.array([0.0, 0.0, 1.0])
    x = _normalize(np.cross(z, up))
    y = np.cross(z, x)
    R = np.stack([x, y, z]).astype(np.float64)
    t = -R @ eye
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(R.astype(np.float32), t.astype(np.float32), float(np.float32(fx)),
                  float(np.float32(fx)), float(width) * 0.5, float(height) * 0.5,
                  int(width), int(height), float(np.float32(znear)))


def stereo_pair(cam: Camera, eye_offset=0.064) -> Tuple[Camera, Camera]:
    """Left/right eyes displaced by -/+ eye_offset/2 along the camera x axis."""
    out = []
    for s in (-0.5, 0.5):
        c = cam.copy()
        # eye centre e = -R^T t; shifting the eye by s*off along camera x changes t by -s*off*e_x
        c.t = (cam.t.astype(np.float64) - np.array([s * eye_offset, 0.0, 0.0])).astype(np.float32)
        out.append(c)
    return out[0], out[1]


def fibonacci_cameras(n_views=8, radius=4.0, **kw) -> List[Camera]:
    """``n_views`` cameras on a Fibonacci lattice of a sphere, all looking at the origin."""
    cams = []
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n_views):
        y = 1.0 - 2.0 * (i + 0.5) / n_views
        r = math.sqrt(max(0.0, 1.0 - y * y))
        th = golden * i
        eye = radius * np.array([r * math.cos(th), y, r * math.sin(th)])
        cams.append(look_at_camera(eye, **kw))
    return cams


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def random_clip_planes(rng: np.random.Generator, n_planes: int, d_range=0.3,
                       layer_bits=0xFFFFFFFF):
    """Planes (n, d, layer_bits) with n uniform on the sphere and d ~ U(-d_range, d_range)."""
    planes = []
    for _ in range(n_planes):
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        d = rng.uniform(-d_range, d_range)
        planes.append((nrm.astype(np.float32), np.float32(d), int(layer_bits)))
    return planes


def uniform_scene(rng: np.random.Generator, n: int, n_layers=2, extent=1.0,
                  log_scale_mu=-3.5, log_scale_sigma=0.5, sh_degree=0,
                  sh_sigma=None) -> Scene:
    """Means uniform in [-extent, extent]^3, layers in contiguous equal blocks.

    With ``sh_sigma`` None and degree 0 the DC coefficient is drawn as
    U(-sqrt(pi), sqrt(pi)), i.e. a base colour uniform in [0, 1].
    """
    means = rng.uniform(-extent, extent, (n, 3)).astype(np.float32)
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    if sh_sigma is None:
        sh = np.zeros((n, K, 3), np.float32)
        sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
        if K > 1:
            sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, K - 1, 3))
    else:
        sh = rng.normal(0.0, sh_sigma, (n, K, 3)).astype(np.float32)
    per = -(-n // n_layers)
    layer = np.minimum(np.arange(n) // per, n_layers - 1).astype(np.uint8)
    return Scene(means, log_scales, quats, opac, sh, layer, sh_degree)


def shell_scene(rng: np.random.Generator, counts: Sequence[int], radii: Sequence[float],
                axes=(1.0, 0.8, 1.25), jitter=0.02, log_scale_mu=-4.5,
                log_scale_sigma=0.7, sh_degree=3, sh_sigma=0.2) -> Scene:
    """Nested jittered ellipsoid shells, one layer per shell (outermost first)."""
    parts = []
    for L, (n, r) in enumerate(zip(counts, radii)):
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rad = r * (1.0 + rng.normal(0.0, jitter, (n, 1)))
        parts.append((d * rad * np.asarray(axes)[None, :]).astype(np.float32))
    means = np.concatenate(parts)
    n = means.shape[0]
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, sh_sigma, (n, K, 3)).astype(np.float32)
    layer = np.concatenate([np.full(c, L, np.uint8) for L, c in enumerate(counts)])
    return Scene(means, log_scales, quats, opac, sh, layer, sh_degree)


# ---------------------------------------------------------------------------
# The five workloads.  ``scale`` shrinks Gaussian counts and image sizes for
# tests that need the same structure at a size the oracle finishes quickly.

def scene_c1(scale: float = 1.0):
    """4,096 Gaussians in 2 layers, SH degree 0, 128x128, both layers on, no plane."""
    rng = np.random.default_rng(config_seed(1))
    n = max(2, int(round(4096 * scale)))
    sc = uniform_scene(rng, n, n_layers=2)
    cam = look_at_camera((0.0, 0.0, 4.0), fov_x_deg=50.0, width=128, height=128)
    return dict(scene=sc, cameras=[cam], layer_mask=0b11, planes=[],
                bg=np.zeros(3, np.float32))


C2_COUNTS = (400_000, 300_000, 250_000, 100_000, 150_000)
C2_RADII = (0.9, 0.75, 0.5, 0.4, 0.3)


def scene_c2(scale: float = 1.0, width: int = 1024, height: int = 1024):
    """1.2M Gaussians on 5 nested shells, SH degree 3, random 5-bit mask, one clip plane."""
    rng = np.random.default_rng(config_seed(2))
    counts = [max(1, int(round(c * scale))) for c in C2_COUNTS]
    sc = shell_scene(rng, counts, C2_RADII)
    mask = int(rng.integers(1, 32))
    planes = random_clip_planes(rng, 1)
    cam = look_at_camera((0.0, 0.0, 4.0), fov_x_deg=50.0, width=width, height=height)
    return dict(scene=sc, cameras=[cam], layer_mask=mask, planes=planes,
                bg=np.zeros(3, np.float32))


def scene_c3(scale: float = 1.0, width: int = 800, height: int = 800, n_views: int = 8):
    """500k Gaussians in 3 shells, 8 Fibonacci cameras, perturbed copy as the target scene."""
    rng = np.random.default_rng(config_seed(3))
    counts = [max(1, int(round(c * scale))) for c in (200_000, 150_000, 150_000)]
    sc = shell_scene(rng, counts, (0.9, 0.6, 0.3))
    tgt = sc.copy()
    tgt.means += rng.normal(0.0, 0.01, tgt.means.shape).astype(np.float32)
    tgt.sh += rng.normal(0.0, 0.05, tgt.sh.shape).astype(np.float32)
    tgt.opacity_logit += rng.normal(0.0, 0.3, tgt.opacity_logit.shape).astype(np.float32)
    cams = fibonacci_cameras(n_views, 4.0, fov_x_deg=50.0, width=width, height=height)
    return dict(scene=sc, target_scene=tgt, cameras=cams, layer_mask=0b111, planes=[],
                bg=np.zeros(3, np.float32))


def scene_c4(scale: float = 1.0, width: int = 2064, height: int = 2208):
    """3M Gaussians (c2 shells x2.5), stereo pair with a 64 mm eye offset."""
    rng = np.random.default_rng(config_seed(4))
    counts = [max(1, int(round(2.5 * c * scale))) for c in C2_COUNTS]
    sc = shell_scene(rng, counts, C2_RADII)
    mask = int(rng.integers(1, 32))
    planes = random_clip_planes(rng, 1)
    centre = look_at_camera((0.0, 0.0, 4.0), fov_x_deg=50.0, width=width, height=height)
    left, right = stereo_pair(centre, 0.064)
    return dict(scene=sc, cameras=[left, right], layer_mask=mask, planes=planes,
                bg=np.zeros(3, np.float32))


def to_half_storage(a: np.ndarray, kind: str) -> np.ndarray:
    """Store float32 values as 16-bit: ``f16`` -> float16, ``bf16`` -> uint16 bit
    patterns rounded to nearest even.  A storage format, not render arithmetic."""
    a = np.ascontiguousarray(a, np.float32)
    if kind == "f16":
        return a.astype(np.float16)
    if kind == "bf16":
        u = a.view(np.uint32).astype(np.uint64)
        rounding = ((u >> 16) & 1) + 0x7FFF
        return ((u + rounding) >> 16).astype(np.uint16)
    raise ValueError(kind)


def from_half_storage(a: np.ndarray, kind: str) -> np.ndarray:
    """Exact widening of 16-bit storage back to float32."""
    if kind == "f16":
        return a.astype(np.float32)
    if kind == "bf16":
        return (a.astype(np.uint32) << 16).view(np.float32)
    raise ValueError(kind)

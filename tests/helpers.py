"""Small scene builders shared by the tests (inputs only, no rendering math)."""
import math

import numpy as np

from synth import Camera, Scene, look_at_camera

Y00 = 0.5 / math.sqrt(math.pi)     # constant real SH of degree 0


def make_scene(means, log_scales, quats=None, opacity_logit=None, rgb=None, layer=None, sh_degree=0,
               sh=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    ls = np.broadcast_to(np.asarray(log_scales, np.float32), (n, 3)).copy()
    q = (np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None
         else np.asarray(quats, np.float32).reshape(n, 4))
    ol = np.zeros(n, np.float32) if opacity_logit is None else np.broadcast_to(
        np.asarray(opacity_logit, np.float32), (n,)).copy()
    K = (sh_degree + 1) ** 2
    if sh is None:
        sh = np.zeros((n, K, 3), np.float32)
        if rgb is not None:
            sh[:, 0, :] = (np.broadcast_to(np.asarray(rgb, np.float64), (n, 3)) - 0.5) / Y00
    sh = np.asarray(sh, np.float32).reshape(n, K, 3)
    lay = np.zeros(n, np.uint8) if layer is None else np.asarray(layer, np.uint8).reshape(n)
    return Scene(means, ls, q, ol, sh, lay, sh_degree)


def axis_camera(z0=4.0, width=33, height=33, fov_x_deg=50.0):
    """Camera on the +z axis at distance z0 looking at the origin."""
    return look_at_camera((0.0, 0.0, z0), fov_x_deg=fov_x_deg, width=width, height=height)


def logit(p):
    return math.log(p / (1.0 - p))


def random_small_scene(seed, n=12, sh_degree=3, n_layers=3, extent=0.5, ls_mu=-2.5, ls_sigma=0.4):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, (n, 3)).astype(np.float32)
    ls = rng.normal(ls_mu, ls_sigma, (n, 3)).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    ol = rng.normal(0.0, 1.0, n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, K, 3)).astype(np.float32)
    layer = rng.integers(0, n_layers, n).astype(np.uint8)
    return Scene(means, ls, q, ol, sh, layer, sh_degree)

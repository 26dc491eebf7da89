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


def branch_scene(seed=7, width=256, height=192, base_n=600):
    """A shell scene plus groups of Gaussians placed in every regime of the
    projection, for pins of the single-precision decision path and the GPU's
    records.  Returns (scene, camera, planes, groups) with groups mapping a
    regime name to the indices of its Gaussians:

      clamp      centres beyond the 1.3x frustum clamp (|x/z| up to 2.2x the
                 half field of view) whose footprint still reaches the frame
      clamp_edge centres within 1e-4 of the clamp boundary
      near       camera depth within 1e-5 .. 1e-3 above the near plane
      needle     one log-scale of -14 (rank-2 covariance before dilation)
      line       two log-scales of -14 (rank 1)
      point      all three log-scales of -14 (the projection is the dilation)
      edge_on    thin discs whose thin axis is perpendicular to the view ray
      tiny_q     quaternions of norm 1e-3 .. 1e-15 (still normal after squaring)
      huge_q     quaternions of norm 1e3 .. 1e15
      opaque     opacity logits of +-30 and colours pushed below zero
    """
    from synth import shell_scene
    rng = np.random.default_rng(seed)
    base = shell_scene(rng, [base_n // 2, base_n - base_n // 2], (0.8, 0.4), sh_degree=3)
    # off-axis eye: the camera rotation has no symmetry, so a transposed
    # rotation somewhere in the projection changes the result
    cam = look_at_camera((0.9, -0.6, 3.8), width=width, height=height)
    Rm, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    tanx = 0.5 * width / cam.fx
    tany = 0.5 * height / cam.fy
    groups = {}
    m, ls, q, ol = [], [], [], []

    def world(pc):                     # camera-space point -> world
        return Rm.T @ (np.asarray(pc, np.float64) - t)

    def add(name, mean, log_scale, quat, logit=1.0):
        groups.setdefault(name, []).append(len(m))
        m.append(mean); ls.append(log_scale); q.append(quat); ol.append(logit)

    def rand_q():
        v = rng.standard_normal(4)
        return v / np.linalg.norm(v)

    for k in range(24):                 # beyond the frustum clamp, large enough to reach the frame
        z = rng.uniform(1.5, 4.0)
        ratio = rng.uniform(1.35, 2.2)
        sx, sy = rng.choice([-1.0, 1.0], 2)
        if k % 3 == 0:
            pc = (sx * ratio * 1.3 * tanx * z, sy * rng.uniform(0, 0.5) * tany * z, z)
        elif k % 3 == 1:
            pc = (sx * rng.uniform(0, 0.5) * tanx * z, sy * ratio * 1.3 * tany * z, z)
        else:
            pc = (sx * ratio * 1.3 * tanx * z, sy * ratio * 1.3 * tany * z, z)
        add("clamp", world(pc), rng.uniform(-0.6, 0.2, 3), rand_q())
    for k in range(12):                 # centres at the clamp boundary
        z = rng.uniform(1.5, 4.0)
        e = rng.uniform(-1e-4, 1e-4)
        pc = ((1.3 + e) * tanx * z * rng.choice([-1.0, 1.0]), rng.uniform(-0.3, 0.3) * tany * z, z)
        add("clamp_edge", world(pc), rng.uniform(-1.0, -0.3, 3), rand_q())
    for k in range(16):                 # just in front of the near plane
        dz = 10.0 ** rng.uniform(-5, -3)
        pc = (rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.05), cam.znear + dz)
        add("near", world(pc), rng.uniform(-6.0, -3.0, 3), rand_q())
    for name, nthin in (("needle", 1), ("line", 2), ("point", 3)):
        for k in range(12):
            l3 = rng.uniform(-3.0, -1.5, 3)
            l3[rng.permutation(3)[:nthin]] = -14.0
            add(name, rng.uniform(-0.5, 0.5, 3) * (1, 1, 0.3), l3, rand_q())
    for k in range(12):                 # edge-on discs: thin axis (local z) perpendicular to the view ray
        pc = np.array([rng.uniform(-0.4, 0.4), rng.uniform(-0.3, 0.3), rng.uniform(3.0, 4.5)])
        mu = world(pc)
        ray = mu - world((0.0, 0.0, 0.0))
        ray /= np.linalg.norm(ray)
        nrm = np.cross(ray, rng.standard_normal(3))
        nrm /= np.linalg.norm(nrm)
        # quaternion rotating e_z onto nrm (half-angle form)
        h = np.array([0.0, 0.0, 1.0]) + nrm
        h /= np.linalg.norm(h)
        axis = np.cross([0.0, 0.0, 1.0], h)
        add("edge_on", mu, (-1.8, -1.8, -14.0), (float(np.dot([0.0, 0.0, 1.0], h)), *axis))
    for k, s in enumerate((1e-3, 1e-5, 1e-8, 1e-10, 1e-12, 1e-15)):
        for j in range(2):
            add("tiny_q", rng.uniform(-0.5, 0.5, 3) * (1, 1, 0.3), rng.uniform(-3.0, -1.5, 3), s * rand_q())
    for k, s in enumerate((1e3, 1e6, 1e9, 1e12, 1e15)):
        for j in range(2):
            add("huge_q", rng.uniform(-0.5, 0.5, 3) * (1, 1, 0.3), rng.uniform(-3.0, -1.5, 3), s * rand_q())
    for lg in (-30.0, -12.0, 12.0, 30.0):
        for j in range(3):
            add("opaque", rng.uniform(-0.5, 0.5, 3) * (1, 1, 0.3), rng.uniform(-3.0, -2.0, 3), rand_q(), lg)
    k_extra = len(m)
    K = (base.sh_degree + 1) ** 2
    sh = rng.normal(0, 0.3, (k_extra, K, 3))
    for i in groups["opaque"]:
        sh[i, 0, :] = -3.0              # base colour well below zero: the colour clamp is active
    lay = rng.integers(0, 2, k_extra).astype(np.uint8)
    n0 = base.n
    groups = {k: np.asarray(v, np.int64) + n0 for k, v in groups.items()}
    sc = Scene(np.concatenate([base.means, np.asarray(m, np.float32)]),
               np.concatenate([base.log_scales, np.asarray(ls, np.float32)]),
               np.concatenate([base.quats, np.asarray(q, np.float32)]),
               np.concatenate([base.opacity_logit, np.asarray(ol, np.float32)]),
               np.concatenate([base.sh, sh.astype(np.float32)]), np.concatenate([base.layer, lay]),
               base.sh_degree)
    planes = [((0.6, 0.0, 0.8), 0.35, 0b10)]
    return sc, cam, planes, groups

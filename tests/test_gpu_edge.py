"""Edge cases of the definition on the GPU against the oracle: degenerate
Gaussians mixed into a normal scene, the largest supported image, a single
pixel, and images whose size is not a multiple of the tile.

Bars as in test_gpu_render: records and integer decisions, tile lists and
ranges bit-exact; every pixel within 1e-5 of the oracle (or its alternative at
a fragile threshold decision)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import Scene
from tests.helpers import branch_scene
from tests.gpu_util import compare_image, compare_lists, compare_records, f64_scene, gpu_render, oracle_stage, read_ws

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _degenerate_scene(seed=31):
    """A shell scene with degenerate Gaussians appended:
    straddling and behind the near plane, centres exactly on the clip plane,
    zero and saturated opacity, needle-thin covariances (one log-scale -14),
    splats larger than the screen, far outside the frustum, and unnormalised
    or near-zero quaternions."""
    rng = np.random.default_rng(seed)
    base = synth.shell_scene(rng, [1500, 1000], (0.8, 0.4), sh_degree=2)
    m, ls, q, ol = [], [], [], []
    cam_z = 4.0
    # near plane at z_cam = 0.2: world z = cam_z - 0.2 = 3.8
    for z in (3.79, 3.8, 3.81, 3.9, 4.5, 6.0):          # around / behind the near plane and behind the camera
        m.append((0.05, -0.03, z)); ls.append((-3.0, -3.0, -3.0)); q.append((1, 0, 0, 0)); ol.append(0.5)
    for x in np.linspace(-0.5, 0.5, 7):                 # on the plane x = 0.1 (normal +x, d = -0.1) and near it
        m.append((0.1 if abs(x) < 0.09 else x, 0.0, 0.3)); ls.append((-4.0, -4.0, -4.0)); q.append((1, 0, 0, 0))
        ol.append(1.0)
    for o in (-30.0, -6.0, 6.0, 30.0):                  # transparent ... saturated
        m.append((rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 0.9)); ls.append((-3.0, -3.0, -3.0))
        q.append((1, 0, 0, 0)); ol.append(o)
    for k in range(6):                                  # needles: one axis far thinner than a pixel
        m.append((rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), 0.5))
        l3 = [-2.5, -2.5, -2.5]; l3[k % 3] = -14.0
        ls.append(tuple(l3)); q.append(tuple(rng.standard_normal(4))); ol.append(2.0)
    for k in range(3):                                  # larger than the screen
        m.append((0.0, 0.0, -0.5 + 0.3 * k)); ls.append((1.5, 1.2, 1.0)); q.append((1, 0, 0, 0)); ol.append(-2.0)
    for p in ((40.0, 0.0, 0.0), (0.0, -40.0, 0.0), (0.0, 0.0, -1e4)):   # far outside / far behind the scene
        m.append(p); ls.append((-1.0, -1.0, -1.0)); q.append((1, 0, 0, 0)); ol.append(1.0)
    for qq in ((1e-30, 0, 0, 0), (0, 0, 0, 3.0), (-2.0, 0.5, 0.5, 0.5)):  # tiny / unnormalised quaternions
        m.append((rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 0.2)); ls.append((-3.5, -3.0, -2.5)); q.append(qq)
        ol.append(0.7)
    k_extra = len(m)
    K = (base.sh_degree + 1) ** 2
    sh = rng.normal(0, 0.3, (k_extra, K, 3)).astype(np.float32)
    lay = rng.integers(0, 2, k_extra).astype(np.uint8)
    sc = Scene(np.concatenate([base.means, np.asarray(m, np.float32)]),
               np.concatenate([base.log_scales, np.asarray(ls, np.float32)]),
               np.concatenate([base.quats, np.asarray(q, np.float32)]),
               np.concatenate([base.opacity_logit, np.asarray(ol, np.float32)]),
               np.concatenate([base.sh, sh]), np.concatenate([base.layer, lay]), base.sh_degree)
    planes = [((1.0, 0.0, 0.0), -0.1, 0b1)]
    cam = synth.look_at_camera((0.0, 0.0, cam_z), width=136, height=120)
    return sc, cam, planes


def _check(sc, cam, mask, planes, bg):
    _, rast, img, al = gpu_render(sc, cam, mask, planes, bg)
    ws = read_ws(rast)
    assert ws["status"].error == 0
    W, H = cam.width, cam.height
    if W * H <= 1 << 20:
        pre, ranges, lst, co = oracle_stage(sc, cam, mask, planes, bg)
        compare_records(ws, pre)
        compare_lists(ws, ranges, lst)
        st = compare_image(img.cpu().numpy(), al.cpu().numpy(), ws["n_contrib"].astype(np.int64), co, TOL)
        assert st["n_bad"] == 0, st
    else:
        # large images: records and lists in full, pixels sampled (uniform plus the centre rows)
        pre = oracle.preprocess(sc, cam, mask, planes, "f32")
        ranges, lst = oracle.bin_tiles(pre)
        compare_records(ws, pre)
        compare_lists(ws, ranges, lst)
        rng = np.random.default_rng(5)
        gx, gy = np.meshgrid(np.arange(W), np.arange(H // 2 - 4, H // 2 + 4))
        xs = np.concatenate([rng.integers(0, W, 16384), gx.ravel()]).astype(np.int32)
        ys = np.concatenate([rng.integers(0, H, 16384), gy.ravel()]).astype(np.int32)
        cp = oracle.composite_pixels(pre, ranges, lst, xs, ys, bg)
        g = img.cpu().numpy()[:, ys, xs].T.astype(np.float64)
        ga = al.cpu().numpy()[ys, xs].astype(np.float64)
        nc = ws["n_contrib"][ys, xs].astype(np.int64)
        e1 = np.maximum(np.abs(g - cp["rgb"]).max(1), np.abs(ga - cp["alpha"]))
        e2 = np.maximum(np.abs(g - cp["alt_rgb"]).max(1), np.abs(ga - cp["alt_alpha"]))
        ok = ((e1 <= TOL) & (nc == cp["ncontrib"])) | ((cp["fragile"] > 0) & (e2 <= TOL) & (nc == cp["alt_ncontrib"]))
        ok |= cp["fragile"] > 1
        assert ok.all(), (int((~ok).sum()), float(e1.max()))
    assert np.isfinite(img.cpu().numpy()).all()
    return pre


def test_degenerate_gaussians():
    sc, cam, planes = _degenerate_scene()
    pre = _check(sc, cam, 0b11, planes, (0.2, 0.3, 0.4))
    extra = slice(2500, sc.n)
    # the near-plane and behind-camera ones are culled exactly as the oracle culls them
    assert pre["vis"][extra].sum() > 0 and (pre["vis"][extra] == 0).sum() > 0


def test_branch_scene_records_lists_and_pixels():
    """The scene whose Gaussians reach every regime of the projection (beyond
    and at the frustum clamp, just in front of the near plane, needle / line /
    point covariances, edge-on discs, quaternions far from unit norm,
    saturated opacities, clamped colours): records bit-exact against the
    oracle's single-precision path (which is itself pinned to the FP64
    definition on the same scene), lists and ranges bit-exact, every pixel
    within 1e-5."""
    sc, cam, planes, groups = branch_scene()
    pre = _check(sc, cam, 0xFFFFFFFF, planes, (0.3, 0.2, 0.1))
    for name, idx in groups.items():
        assert pre["vis"][idx].sum() > 0, name


@pytest.mark.parametrize("W,H", [(1, 1), (17, 1), (1, 33), (4096, 4096), (4096, 16), (31, 4095)])
def test_image_sizes(W, H):
    """One pixel, single rows and columns, ragged tiles and the largest image
    (4096 x 4096, the binning's limit)."""
    rng = np.random.default_rng(W * 7 + H)
    sc = synth.shell_scene(rng, [3000, 2000], (0.8, 0.45), sh_degree=1)
    cam = synth.look_at_camera((0.2, -0.1, 3.4), width=W, height=H)
    _check(sc, cam, 0b11, [], (0.0, 0.5, 1.0))


def _plane_scene(rng, n, depths, sh_degree=1):
    """n Gaussians with means spread in x, y and their z from `depths`."""
    m = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), depths], 1).astype(np.float32)
    K = (sh_degree + 1) ** 2
    return Scene(m, rng.normal(-4.0, 0.4, (n, 3)).astype(np.float32),
                 rng.standard_normal((n, 4)).astype(np.float32), rng.normal(0.0, 1.5, n).astype(np.float32),
                 rng.normal(0, 0.3, (n, K, 3)).astype(np.float32), rng.integers(0, 2, n).astype(np.uint8), sh_degree)


@pytest.mark.parametrize("kind", ["equal", "wide"])
def test_depth_sort_digit_counts(kind):
    """The depth sort runs one digit kernel per byte below the highest bit
    where the smallest and largest key differ: all depths equal (only the
    first, compacting kernel runs; ties stay in index order) and depths from
    0.25 to 1000 (the keys differ in the top byte: all four run).  Several
    2048-item sort tiles and a ragged last tile; lists bit-exact."""
    rng = np.random.default_rng(17 if kind == "equal" else 18)
    n = 9000
    # camera on the +z axis looking at the origin: the depth of (x, y, z) is exactly 3 - z
    if kind == "equal":
        z = np.zeros(n)
    else:
        z = 3.0 - np.exp(rng.uniform(np.log(0.25), np.log(1000.0), n))
    sc = _plane_scene(rng, n, z)
    cam = synth.look_at_camera((0.0, 0.0, 3.0), width=96, height=80)
    pre = _check(sc, cam, 0b11, [], (0.1, 0.1, 0.1))
    d = pre["depth_f32"][pre["vis"] > 0].view(np.uint32) if "depth_f32" in pre else None
    if d is not None:
        span = int(d.min() ^ d.max())
        assert (span == 0) if kind == "equal" else (span >> 24) != 0


def _heavy_scene(seed=23):
    """A dense scene seen through a small image: most visible Gaussians cover
    most tiles, so tile lists run to many thousands of positions (walks over
    dozens of 256-position checkpoint segments), half the pixels stop early
    and half walk their whole list."""
    rng = np.random.default_rng(seed)
    sc = synth.shell_scene(rng, [14000, 10000], (0.8, 0.45), sh_degree=2, log_scale_mu=-2.2,
                           log_scale_sigma=0.4)
    sc.opacity_logit = (sc.opacity_logit - 4.0).astype(np.float32)     # mostly faint splats: long walks
    cam = synth.look_at_camera((0.3, 0.2, 3.2), width=96, height=64, fov_x_deg=45.0)
    return sc, cam


def test_long_lists_forward():
    sc, cam = _heavy_scene()
    _, rast, img, al = gpu_render(sc, cam, 0b11, [], (0.3, 0.2, 0.1))
    ws = read_ws(rast)
    assert ws["status"].error == 0
    pre, ranges, lst, co = oracle_stage(sc, cam, 0b11, [], (0.3, 0.2, 0.1))
    lens = ranges[:, 1] - ranges[:, 0]
    assert (lens >= 4096).sum() >= 4 and (lens < 4096).sum() >= 1, lens
    compare_records(ws, pre)
    compare_lists(ws, ranges, lst)
    st = compare_image(img.cpu().numpy(), al.cpu().numpy(), ws["n_contrib"].astype(np.int64), co, TOL)
    assert st["n_bad"] == 0, st
    # some pixels stop early and some walk their whole list
    nc = ws["n_contrib"].astype(np.int64)
    assert (co["T"] < 1e-3).any() and (co["T"] > 1e-3).any()
    assert nc.max() > 4096


def test_long_lists_backward():
    """The backward walks back through dozens of checkpoint segments per
    pixel: gradients within the field-normalised 1e-5 bar of the oracle.  These
    splats cover most of the image, so nearly every one meets some pixel with
    a threshold decision within rounding (fragile); the upstream gradient is
    zero at those pixels, on both sides, and every Gaussian is compared."""
    sc, cam = _heavy_scene()
    bg = (0.3, 0.2, 0.1)
    ds, rast, img, al = gpu_render(sc, cam, 0b11, [], bg)
    pre, ranges, lst, co = oracle_stage(sc, cam, 0b11, [], bg)
    rng = np.random.default_rng(4)
    dimg = rng.standard_normal((3, cam.height, cam.width)).astype(np.float32)
    dal = rng.standard_normal((cam.height, cam.width)).astype(np.float32)
    fr = co["fragile"] > 0
    assert fr.mean() < 0.2
    dimg[:, fr] = 0.0
    dal[fr] = 0.0
    g = rast.backward(ds, cam, bg, torch.from_numpy(dimg).cuda(), torch.from_numpy(dal).cuda())
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    cb = oracle.composite_backward(pre, ranges, lst, bg, dimg, dal)
    ref = oracle.chain(f64_scene(sc), cam, pre["vis"], cb["rec_grad"])
    ok = cb["contrib_max"] > 0
    assert ok.sum() > 1000
    for f in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        a = g[f].reshape(sc.n, -1)[ok].astype(np.float64)
        b = ref[f].reshape(sc.n, -1)[ok]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), f

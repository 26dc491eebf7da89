"""Pins of the oracle's tile binning and front-to-back compositing (Sec. 3.3:
Gaussians sorted relative to the camera and rendered as splats; Sec. 1 and
Sec. 5: layers shown alone or together, cut, and never overriding each other)."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import axis_camera, logit, make_scene, random_small_scene

BG = np.array([0.1, 0.2, 0.3])


def _render(sc, cam, **kw):
    return oracle.render(sc, cam, bg=kw.pop("bg", BG), **kw)


def test_single_isotropic_splat_at_pixel_centre():
    z0, s, o = 4.0, 0.02, 0.6
    cam = axis_camera(z0, 33, 33)
    rgb = np.array([0.9, 0.5, 0.25])
    sc = make_scene([[0, 0, 0]], math.log(s), rgb=rgb, opacity_logit=logit(o))
    r = _render(sc, cam)
    s = math.exp(float(sc.log_scales[0, 0]))
    o = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    rgb = (sc.sh[0, 0].astype(np.float64) * (0.5 / math.sqrt(math.pi))) + 0.5
    sig2 = (cam.fx * s / z0) ** 2 + 0.3
    # centre pixel: d = 0, alpha = o
    assert np.allclose(r["image"][:, 16, 16], o * rgb + (1 - o) * BG, atol=1e-14)
    assert abs(r["alpha"][16, 16] - o) < 1e-14
    # one pixel to the right: alpha = o exp(-1/(2 sigma'^2))
    a1 = o * math.exp(-0.5 / sig2)
    assert np.allclose(r["image"][:, 16, 17], a1 * rgb + (1 - a1) * BG, atol=1e-14)
    # diagonal neighbour: alpha = o exp(-2/(2 sigma'^2))
    a2 = o * math.exp(-1.0 / sig2)
    assert abs(r["alpha"][15, 15] - a2) < 1e-14


def test_two_splat_ordering_and_swap():
    cam = axis_camera(4.0, 33, 33)
    c1, c2 = [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]
    o1, o2 = 0.7, 0.4
    sc = make_scene([[0, 0, 0.5], [0, 0, -0.5]], math.log(0.05), rgb=[c1, c2],
                    opacity_logit=[logit(o1), logit(o2)])
    r = _render(sc, cam)
    o1 = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    o2 = 1 / (1 + math.exp(-float(sc.opacity_logit[1])))
    k1 = sc.sh[0, 0].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    k2 = sc.sh[1, 0].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    want = o1 * k1 + (1 - o1) * o2 * k2 + (1 - o1) * (1 - o2) * BG        # splat 0 is nearer
    assert np.allclose(r["image"][:, 16, 16], want, atol=1e-14)
    sc.means[:, 2] = sc.means[::-1, 2]                                     # swap depths
    r = _render(sc, cam)
    want = o2 * k2 + (1 - o2) * o1 * k1 + (1 - o1) * (1 - o2) * BG
    assert np.allclose(r["image"][:, 16, 16], want, atol=1e-14)


def test_equal_depth_orders_by_index():
    cam = axis_camera(4.0, 33, 33)
    sc = make_scene([[0, 0, 0], [0, 0, 0]], math.log(0.05), rgb=[[1, 0, 0], [0, 1, 0]],
                    opacity_logit=[logit(0.5), logit(0.5)])
    r = _render(sc, cam)
    t = (16 // 16) * 3 + 16 // 16
    lo, hi = r["ranges"][t]
    assert list(r["list"][lo:hi]) == [0, 1]
    o = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    k = sc.sh[:, 0].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    assert np.allclose(r["image"][:, 16, 16], o * k[0] + (1 - o) * o * k[1] + (1 - o) ** 2 * BG, atol=1e-14)


def test_transmittance_invariant_white_on_white():
    # every colour 1 and background 1: sum_i a_i T_i + T_N = 1 at every pixel
    w = synth.scene_c1(scale=0.25)
    sc = w["scene"]
    sc.sh[:] = 0.0
    sc.sh[:, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))
    r = oracle.render(sc, w["cameras"][0], bg=np.ones(3))
    c = float(sc.sh[0, 0, 0]) * (0.5 / math.sqrt(math.pi)) + 0.5    # 1 up to float32 storage of the SH
    # image = c (1 - T) + T exactly when every colour is c
    assert np.abs(r["image"] - (c * r["alpha"] + (1 - r["alpha"]))).max() < 1e-13
    assert abs(c - 1) < 1e-7 and r["alpha"].max() > 0.9


def test_transmittance_is_product_over_blended_splats():
    sc = random_small_scene(8, n=10, sh_degree=0)
    cam = axis_camera(4.0, 32, 32)
    r = oracle.render(sc, cam, bg=np.zeros(3))
    # with rgb = 1 and bg = 0 the image is 1 - T
    sc2 = sc.copy()
    sc2.sh[:, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))
    r2 = oracle.render(sc2, cam, bg=np.zeros(3))
    c = float(sc2.sh[0, 0, 0]) * (0.5 / math.sqrt(math.pi)) + 0.5
    assert np.abs(r2["image"][0] - c * r["alpha"]).max() < 1e-13
    assert np.abs(r2["image"][0] - c * (1 - r2["T"])).max() < 1e-13


@pytest.mark.parametrize("alpha,k", [(0.5, 30), (0.3, 10), (0.9, 8), (0.99, 5)])
def test_early_stop_count(alpha, k):
    # k identical splats stacked on the axis: splat j (0-based) is blended iff
    # (1-a)^(j+1) >= 1e-4, so the count is min(k, floor(ln 1e-4 / ln(1-a))).
    cam = axis_camera(4.0, 33, 33)
    zs = np.linspace(0.5, -0.5, k)
    sc = make_scene([[0, 0, z] for z in zs], math.log(0.05), rgb=[0.5, 0.5, 0.5],
                    opacity_logit=logit(alpha) if alpha < 0.99 else 10.0)
    r = _render(sc, cam)
    a = min(0.99, 1 / (1 + math.exp(-float(sc.opacity_logit[0]))))
    want = min(k, math.floor(math.log(1e-4) / math.log(1 - a)))
    assert r["ncontrib"][16, 16] == want
    assert abs(r["T"][16, 16] - (1 - a) ** want) < 1e-14


def test_alpha_threshold_and_clamp():
    cam = axis_camera(4.0, 33, 33)
    lo = (1 / 255) * (1 - 1e-3)
    hi = (1 / 255) * (1 + 1e-3)
    for o, blended in ((lo, False), (hi, True)):
        sc = make_scene([[0, 0, 0]], math.log(0.02), rgb=[1, 1, 1], opacity_logit=logit(o))
        r = _render(sc, cam, bg=np.zeros(3))
        assert (r["alpha"][16, 16] > 0) == blended
        assert r["ncontrib"][16, 16] == (1 if blended else 0)
    sc = make_scene([[0, 0, 0]], math.log(0.02), rgb=[1, 1, 1], opacity_logit=12.0)
    r = _render(sc, cam, bg=np.zeros(3))
    assert r["alpha"][16, 16] == 0.99


def test_mask_zero_is_background():
    w = synth.scene_c1(scale=0.25)
    r = oracle.render(w["scene"], w["cameras"][0], layer_mask=0, bg=BG)
    assert np.array_equal(r["image"], np.broadcast_to(BG[:, None, None], r["image"].shape))
    assert np.all(r["alpha"] == 0)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_masking_a_layer_equals_deleting_it(precision):
    sc = random_small_scene(9, n=40, n_layers=3)
    cam = axis_camera(3.0, 48, 40)
    for mask in (0b001, 0b011, 0b101, 0b110):
        a = oracle.render(sc, cam, layer_mask=mask, bg=BG, precision=precision)
        keep = np.array([(mask >> int(l)) & 1 for l in sc.layer], bool)
        b = oracle.render(sc.subset(keep), cam, layer_mask=0xFFFFFFFF, bg=BG, precision=precision)
        assert np.array_equal(a["image"], b["image"])
        assert np.array_equal(a["alpha"], b["alpha"])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_clipping_equals_deleting_the_cut_gaussians(precision):
    sc = random_small_scene(10, n=40, n_layers=3)
    cam = axis_camera(3.0, 48, 48)
    rng = np.random.default_rng(11)
    planes = synth.random_clip_planes(rng, 2, 0.2, layer_bits=0b011)
    a = oracle.render(sc, cam, planes=planes, bg=BG, precision=precision)
    mu = sc.means.astype(np.float64)
    keep = np.ones(sc.n, bool)
    for nrm, d, bits in planes:
        dist = mu @ nrm.astype(np.float64) + float(d)
        inl = np.array([(bits >> int(l)) & 1 for l in sc.layer], bool)
        keep &= ~(inl & (dist < 0))
    b = oracle.render(sc.subset(keep), cam, bg=BG, precision=precision)
    assert np.array_equal(a["image"], b["image"])


def test_sorted_lists_match_lexsort():
    sc = random_small_scene(12, n=60, extent=0.6)
    cam = axis_camera(3.0, 64, 48)
    for prec in ("f64", "f32"):
        pre = oracle.preprocess(sc, cam, precision=prec)
        ranges, lst = oracle.bin_tiles(pre)
        Tx = (64 + 15) // 16
        tiles, depth, idx = [], [], []
        for i in np.nonzero(pre["vis"])[0]:
            x0, y0, x1, y1 = pre["rect"][i]
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    tiles.append(ty * Tx + tx)
                    depth.append(pre["depth"][i])
                    idx.append(i)
        order = np.lexsort((idx, depth, tiles))
        assert np.array_equal(lst, np.array(idx)[order])
        t_sorted = np.array(tiles)[order]
        for t in range(ranges.shape[0]):
            sel = np.nonzero(t_sorted == t)[0]
            if sel.size:
                assert ranges[t, 0] == sel[0] and ranges[t, 1] == sel[-1] + 1
            else:
                assert ranges[t, 0] == ranges[t, 1]


@pytest.mark.parametrize("seed", [13, 14, 15])
def test_tiled_render_equals_brute_force(seed):
    # Brute force: every visible Gaussian at every pixel in (depth, index) order.
    # Pixels where some splat has alpha >= 1/255 outside its tile rectangle are
    # where the tiled render legitimately truncates; they are excluded.
    sc = random_small_scene(seed, n=8, sh_degree=1, extent=0.4, ls_mu=-2.8)
    cam = axis_camera(3.0, 32, 32)
    r = oracle.render(sc, cam, bg=BG)
    bf = oracle.composite_bruteforce(r["pre"], bg=BG)
    pre = r["pre"]
    trunc = np.zeros((32, 32), bool)
    ys, xs = np.mgrid[0:32, 0:32] + 0.5
    for i in np.nonzero(pre["vis"])[0]:
        dx, dy = xs - pre["u"][i], ys - pre["v"][i]
        p = dx + pre["beta"][i] * dy
        a = pre["opac"][i] * np.exp2(pre["A2"][i] * p * p + pre["G2"][i] * dy * dy)
        x0, y0, x1, y1 = pre["rect"][i]
        inside = np.zeros((32, 32), bool)
        inside[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
        trunc |= (a >= 1 / 255) & ~inside
    ok = ~trunc
    assert ok.mean() > 0.5
    assert np.abs(r["image"] - bf["image"])[:, ok].max() < 1e-13
    assert np.abs(r["alpha"] - bf["alpha"])[ok].max() < 1e-13


def test_fragile_alternative_flips_first_decision():
    # a splat whose alpha sits within the relative margin of 1/255 at the centre
    cam = axis_camera(4.0, 33, 33)
    o = (1 / 255) * (1 + 2e-6)
    sc = make_scene([[0, 0, 0]], math.log(0.02), rgb=[1, 1, 1], opacity_logit=logit(o))
    r = _render(sc, cam, bg=np.zeros(3))
    assert r["fragile"][16, 16] == 1
    assert r["ncontrib"][16, 16] == 1 and r["alt_ncontrib"][16, 16] == 0
    assert r["alt_alpha"][16, 16] == 0.0


def test_prune_definition():
    cm = np.array([0.0, 0.004999, 0.005, 0.7])
    keep, k = oracle.prune(cm, 0.005)
    assert list(keep) == [0, 0, 1, 1] and k == 2


def _ragged_frame(seed):
    # 40 Gaussians over a 56x40 frame: 4x3 tiles, the last column and row ragged
    sc = random_small_scene(seed, n=40, sh_degree=1, extent=0.45, ls_mu=-2.6)
    cam = axis_camera(2.6, 56, 40)
    pre = oracle.preprocess(sc, cam)
    ranges, lst = oracle.bin_tiles(pre)
    return sc, cam, pre, ranges, lst


@pytest.mark.parametrize("seed", [21, 22])
def test_sampled_pixels_equal_the_full_composite(seed):
    # The sampled compositor (used to check large frames one pixel at a time) is
    # the full compositor restricted to the listed pixels: every output, in any
    # order of the samples, bit for bit.
    _, _, pre, ranges, lst = _ragged_frame(seed)
    co = oracle.composite(pre, ranges, lst, BG)
    H, W = co["alpha"].shape
    ys, xs = np.divmod(np.random.default_rng(seed).permutation(W * H), W)
    cp = oracle.composite_pixels(pre, ranges, lst, xs, ys, BG)
    assert co["ncontrib"].max() > 1 and (co["alpha"] > 0).mean() > 0.3
    assert np.array_equal(cp["rgb"], co["image"][:, ys, xs].T)
    assert np.array_equal(cp["alpha"], co["alpha"][ys, xs])
    assert np.array_equal(cp["ncontrib"], co["ncontrib"][ys, xs])
    assert np.array_equal(cp["fragile"], co["fragile"][ys, xs])
    assert np.array_equal(cp["alt_rgb"], co["alt_image"][:, ys, xs].T)
    assert np.array_equal(cp["alt_alpha"], co["alt_alpha"][ys, xs])
    assert np.array_equal(cp["alt_ncontrib"], co["alt_ncontrib"][ys, xs])


@pytest.mark.parametrize("seed", [23, 24])
def test_tile_restricted_backward(seed):
    # The backward restricted to some tiles (how large frames are checked patch
    # by patch): with every tile marked it is the unrestricted pass; with dL zero
    # outside the marked tiles the record gradients are those of the full pass
    # bit for bit (the skipped tiles only add zeros); blend weights only count
    # the marked tiles, so they never exceed the full pass's and equal them for
    # a Gaussian whose whole rectangle is marked.
    _, _, pre, ranges, lst = _ragged_frame(seed)
    H, W = pre["H"], pre["W"]
    Tx, Ty = (W + 15) // 16, (H + 15) // 16
    rng = np.random.default_rng(seed)
    dimg = rng.standard_normal((3, H, W))
    dal = rng.standard_normal((H, W))
    full = oracle.composite_backward(pre, ranges, lst, BG, dimg, dal)
    ones = oracle.composite_backward(pre, ranges, lst, BG, dimg, dal, np.ones(Tx * Ty, np.uint8))
    for k in ("rec_grad", "contrib_sum", "contrib_max", "touched_fragile"):
        assert np.array_equal(ones[k], full[k]), k
    tm2 = np.zeros((Ty, Tx), np.uint8)
    tm2[:2, 1:3] = 1
    inside = np.kron(tm2, np.ones((16, 16), np.uint8))[:H, :W] > 0
    dimg_m, dal_m = dimg * inside, dal * inside
    full_m = oracle.composite_backward(pre, ranges, lst, BG, dimg_m, dal_m)
    part = oracle.composite_backward(pre, ranges, lst, BG, dimg_m, dal_m, tm2.reshape(-1))
    assert np.abs(full_m["rec_grad"]).max() > 0
    assert np.array_equal(part["rec_grad"], full_m["rec_grad"])
    assert np.all(part["contrib_max"] <= full["contrib_max"])
    assert np.all(part["contrib_sum"] <= full["contrib_sum"] * (1 + 1e-12))
    vis = np.nonzero(pre["vis"])[0]
    whole = [i for i in vis if tm2[pre["rect"][i][1]:pre["rect"][i][3], pre["rect"][i][0]:pre["rect"][i][2]].all()]
    assert len(whole) >= 1
    assert np.array_equal(part["contrib_max"][whole], full["contrib_max"][whole])
    assert np.allclose(part["contrib_sum"][whole], full["contrib_sum"][whole], rtol=1e-12, atol=0)


def test_oracle_rejects_out_of_frame_inputs():
    # the C oracle does no bounds checks of its own: its wrappers refuse what would
    # index outside the frame or the tile array
    _, _, pre, ranges, lst = _ragged_frame(21)
    with pytest.raises(ValueError):
        oracle.composite_pixels(pre, ranges, lst, np.array([pre["W"]]), np.array([0]), BG)
    with pytest.raises(ValueError):
        oracle.composite_pixels(pre, ranges, lst, np.array([0]), np.array([-1]), BG)
    with pytest.raises(ValueError):
        oracle.composite_backward(pre, ranges, lst, BG, np.zeros((3, pre["H"], pre["W"])), None,
                                  np.ones(ranges.shape[0] - 1, np.uint8))

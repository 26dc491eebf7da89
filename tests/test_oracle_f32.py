"""Pins of the oracle's single-precision decision path against its FP64
definition: the same projection, with integer decisions (culls, radius, tile
rectangle, depth key) taken in IEEE single precision in a fixed order.

The single-precision record fields of EVERY visible Gaussian must lie within a
first-order forward error bound of the FP64 definition.  The bound is derived
per Gaussian from the magnitudes of the quantities the projection combines
(standard floating-point error analysis, unit roundoff u = 2^-24): where the
projection cancels (a centre close to the near plane, an ill-conditioned 2D
covariance, a thin covariance seen edge-on) the bound widens by exactly the
factor the cancellation costs, and nowhere else.  The scenes reach every branch:
the frustum clamp (and its boundary), the near plane, needle / line / point
covariances before the dilation, edge-on discs, quaternions far from unit norm,
saturated opacities and clamped colours.  A test plants mistakes in a scratch
copy of the oracle and requires this pin to catch each of them."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth
from tests.helpers import branch_scene

U = 2.0 ** -24          # unit roundoff of IEEE binary32, round to nearest
SAFETY = 2.0            # first-order bound; the factor covers the second-order terms


def test_expf32_error_bound():
    xs = np.concatenate([np.linspace(-80, 80, 20001), np.linspace(-1, 1, 2001),
                         np.random.default_rng(0).uniform(-20, 20, 5000)]).astype(np.float32)
    got = oracle.expf32(xs).astype(np.float64)
    want = np.exp(xs.astype(np.float64))
    rel = np.abs(got - want) / want
    assert rel.max() < 2.0 ** -21          # within 4 units in the last place
    assert oracle.expf32([0.0])[0] == 1.0


def test_expf32_saturates_outside_range():
    assert oracle.expf32([200.0])[0] == oracle.expf32([80.0])[0]
    assert oracle.expf32([-200.0])[0] == oracle.expf32([-80.0])[0] > 0


# --------------------------------------------------------------------------- error bounds

def f32_error_bounds(sc, cam, planes):
    """Per-Gaussian first-order bounds on |f32 - f64| of every record field
    of the single-precision projection, and the margins of its decisions.

    Error model (each step of the f32 path is one rounded IEEE operation):
      scales  s = exp(l) within 8u relative (the 4-ulp exponential);
      q/|q|   each component within 4u relative (4 products and sums of
              squares, one square root, one division);
      R(q)    every entry within 21u absolute (|x y| + |w z| <= 1/2 on the
              unit sphere);
      M = R S column l within 21u s_l (every component) + 9u |r_l| s_l;
      Sigma = M M^T with 3u per product-sum;
      p = W mu + t within 4u (|W||mu| + |t|) per coordinate;
      x/z     within 4u |W_x||mu|/z + |x/z| (rel(z) + u), the clamp is
              1-Lipschitz and its limit carries 3u;
      J, T=JW from those, with 2u per product-sum; Sigma' = T Sigma T^T + 0.3 I
              within |dT||Sigma||T| + |T||Sigma||dT| + sum_l of the moves of
              (T m_l)(T m_l)^T + 6u |T||Sigma||T|^T, plus u for the dilation;
      det, A2, beta, G2, the radius and the rectangle from those by the
              usual rules for products, quotients and square roots.
    Magnitudes are evaluated in double precision from scipy's rotations, not
    from the oracle."""
    m = sc.means.astype(np.float64)
    s = np.exp(sc.log_scales.astype(np.float64))
    q = sc.quats.astype(np.float64)
    n = sc.n
    Rq = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()           # scipy: (x, y, z, w)
    Sig = np.einsum("nij,nj,nkj->nik", Rq, s * s, Rq)
    W = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    p = m @ W.T + t
    pabs = np.abs(m) @ np.abs(W).T + np.abs(t)
    x, y, z = p[:, 0], p[:, 1], np.where(p[:, 2] > 0, p[:, 2], np.inf)
    rel_z = 4 * U * pabs[:, 2] / z
    ix, iy = x / z, y / z
    d_ix = 4 * U * pabs[:, 0] / z + np.abs(ix) * (rel_z + U)
    d_iy = 4 * U * pabs[:, 1] / z + np.abs(iy) * (rel_z + U)
    limx = 1.3 * (0.5 * cam.width / fx)
    limy = 1.3 * (0.5 * cam.height / fy)
    cxz, cyz = np.clip(ix, -limx, limx), np.clip(iy, -limy, limy)
    d_cx, d_cy = d_ix + 3 * U * limx, d_iy + 3 * U * limy
    j00, j02, j11, j12 = fx / z, -fx * cxz / z, fy / z, -fy * cyz / z
    d_j00, d_j11 = np.abs(j00) * (rel_z + U), np.abs(j11) * (rel_z + U)
    d_j02 = fx * d_cx / z + np.abs(j02) * (rel_z + 2 * U)
    d_j12 = fy * d_cy / z + np.abs(j12) * (rel_z + 2 * U)
    T = np.stack([j00[:, None] * W[0] + j02[:, None] * W[2], j11[:, None] * W[1] + j12[:, None] * W[2]], 1)
    Tabs = np.stack([np.abs(j00)[:, None] * np.abs(W[0]) + np.abs(j02)[:, None] * np.abs(W[2]),
                     np.abs(j11)[:, None] * np.abs(W[1]) + np.abs(j12)[:, None] * np.abs(W[2])], 1)
    dT = np.stack([d_j00[:, None] * np.abs(W[0]) + d_j02[:, None] * np.abs(W[2]),
                   d_j11[:, None] * np.abs(W[1]) + d_j12[:, None] * np.abs(W[2])], 1) + 2 * U * Tabs
    aS = np.abs(Sig)
    C = np.einsum("naj,njk,nbk->nab", T, Sig, T) + 0.3 * np.eye(2)
    Cabs = np.einsum("naj,njk,nbk->nab", Tabs, aS, Tabs)
    # rotation and scale errors of M = R S: column l of M moves by at most
    # 21u s_l in every component (rotation) and 9u |r_l| s_l (scale), so its
    # image under T moves by 21u s_l sum|T_a| + 9u s_l (|T||R|)_al
    rs = Tabs.sum(2)                                                    # [n, 2]
    A = np.einsum("naj,njl->nal", Tabs, np.abs(Rq))                     # [n, 2, 3]
    s2 = s * s
    dTM = 21 * U * rs[:, :, None] + 9 * U * A                           # [n, 2, 3] per unit s_l
    dC = (np.einsum("naj,njk,nbk->nab", dT, aS, Tabs) + np.einsum("naj,njk,nbk->nab", Tabs, aS, dT)
          + np.einsum("nl,nal,nbl->nab", s2, dTM, A) + np.einsum("nl,nal,nbl->nab", s2, A, dTM)
          + 3 * U * np.einsum("nl,nal,nbl->nab", s2, A, A) + 6 * U * Cabs + U * np.abs(C))
    c00, c01, c11 = C[:, 0, 0], C[:, 0, 1], C[:, 1, 1]
    e00, e01, e11 = dC[:, 0, 0], dC[:, 0, 1], dC[:, 1, 1]
    det = c00 * c11 - c01 * c01
    d_det = e00 * c11 + c00 * e11 + 2 * np.abs(c01) * e01 + 3 * U * (c00 * c11 + c01 * c01)
    nhl = 0.5 * math.log2(math.e)
    A2, beta, G2 = -nhl * c11 / det, -c01 / c11, -nhl / c11
    b = {}
    b["A2"] = np.abs(A2) * (e11 / c11 + d_det / det + 3 * U)
    b["beta"] = e01 / c11 + np.abs(c01) * e11 / c11 ** 2 + U * np.abs(beta)
    b["G2"] = np.abs(G2) * (e11 / c11 + 2 * U)
    b["u"] = fx * d_ix + U * fx * np.abs(ix) + U * np.abs(fx * ix + cx)
    b["v"] = fy * d_iy + U * fy * np.abs(iy) + U * np.abs(fy * iy + cy)
    b["depth"] = 4 * U * pabs[:, 2]
    o = 1.0 / (1.0 + np.exp(-sc.opacity_logit.astype(np.float64)))
    b["opac"] = 10 * U * o
    # colour: direction from the camera centre, SH basis (|Y_k| and the sums of
    # the absolute values of its terms are below 3.5 for degree <= 3), the sum
    campos = -W.T @ t
    d_cam = 3 * U * (np.abs(W) * np.abs(t)[:, None]).sum(0)
    dv = m - campos
    dn = np.linalg.norm(dv, axis=1)
    d_dir = 2 * (d_cam.max() + U * np.abs(dv).max(1)) / dn + 4 * U
    K = (sc.sh_degree + 1) ** 2
    deg_k = np.floor(np.sqrt(np.arange(K))).astype(np.int64)
    shabs = np.abs(sc.sh.astype(np.float64))                            # [n, K, 3]
    db = 3 * 3.5 * deg_k[None, :] * d_dir[:, None] + 28 * U
    acc_abs = (3.5 * shabs).sum(1) + 0.5
    b["rgb"] = (shabs * db[:, :, None]).sum(1) + (K + 2) * U * acc_abs
    # radius: ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det))
    mid = 0.5 * (c00 + c11)
    d_mid = 0.5 * (e00 + e11) + U * mid
    xd = mid * mid - det
    d_xd = 2 * mid * d_mid + d_det + 2 * U * (mid * mid + np.abs(det))
    disc = np.maximum(0.1, xd)
    d_disc = d_xd + U * 0.1
    sq = np.sqrt(disc)
    lam = mid + sq
    d_lam = d_mid + d_disc / (2 * sq) + U * sq + U * lam
    r3 = 3 * np.sqrt(lam)
    d_r3 = 3 * (d_lam / (2 * np.sqrt(lam)) + U * np.sqrt(lam)) + U * r3
    for k in b:
        b[k] = SAFETY * b[k]
    d_r3 = SAFETY * d_r3
    margins = {}
    margins["radius"] = np.abs(r3 - np.round(r3)) > d_r3
    r = np.ceil(r3)
    ok_rect = np.ones(n, bool)
    for c, dc in ((fx * ix + cx, b["u"]), (fy * iy + cy, b["v"])):
        for e in ((c - r) / 16.0, (c + r + 15.0) / 16.0):
            ok_rect &= np.abs(e - np.round(e)) > dc / 16.0 + 2 * U * np.abs(e) + 1e-12
    margins["rect"] = ok_rect & margins["radius"]
    # culls: the near plane and every clip plane of the Gaussian's layer
    ok_cull = np.abs(p[:, 2] - cam.znear) > 2 * b["depth"] + U * cam.znear
    for nrm, dd, bits in planes:
        nv = np.asarray(nrm, np.float32).astype(np.float64)
        dist = m @ nv + float(np.float32(dd))
        dd_abs = 4 * U * (np.abs(m) @ np.abs(nv) + abs(float(dd)))
        applies = ((int(bits) >> sc.layer.astype(np.int64)) & 1) > 0
        ok_cull &= ~applies | (np.abs(dist) > SAFETY * dd_abs)
    margins["cull"] = ok_cull & margins["rect"]
    return b, margins


def check_f32_against_f64(sc, cam, mask, planes):
    """Every single-precision record field of every visible Gaussian within
    its bound of the FP64 definition; integer decisions equal wherever the
    FP64 quantity is farther from the decision boundary than the bound."""
    p64 = oracle.preprocess(sc, cam, mask, planes, "f64")
    p32 = oracle.preprocess(sc, cam, mask, planes, "f32")
    b, mg = f32_error_bounds(sc, cam, planes)
    clear = mg["cull"]
    assert np.array_equal(p64["vis"][clear], p32["vis"][clear]), "culls differ away from their boundaries"
    both = (p64["vis"] > 0) & (p32["vis"] > 0)
    worst = {}
    for k in ("u", "v", "depth", "A2", "beta", "G2", "opac"):
        ratio = np.abs(p32[k][both] - p64[k][both]) / b[k][both]
        worst[k] = float(ratio.max())
        assert worst[k] <= 1.0, (k, worst[k], int(np.nonzero(both)[0][ratio.argmax()]))
    ratio = np.abs(p32["rgb"][both] - p64["rgb"][both]) / b["rgb"][both]
    worst["rgb"] = float(ratio.max())
    assert worst["rgb"] <= 1.0, ("rgb", worst["rgb"])
    ok = both & mg["radius"]
    assert np.array_equal(p64["radius"][ok], p32["radius"][ok]), "radius"
    ok = both & mg["rect"]
    assert np.array_equal(p64["rect"][ok], p32["rect"][ok]), "rect"
    return dict(p64=p64, p32=p32, bounds=b, margins=mg, both=both, worst=worst)


def _scenes():
    w1 = synth.scene_c1()
    w2 = synth.scene_c2(scale=0.01, width=256, height=256)
    sc, cam, planes, groups = branch_scene()
    return {"c1": (w1["scene"], w1["cameras"][0], w1["layer_mask"], w1["planes"]),
            "c2_small": (w2["scene"], w2["cameras"][0], w2["layer_mask"], w2["planes"]),
            "branches": (sc, cam, 0xFFFFFFFF, planes)}


@pytest.mark.parametrize("which", ["c1", "c2_small", "branches"])
def test_f32_path_within_error_bound_of_f64_definition(which):
    sc, cam, mask, planes = _scenes()[which]
    r = check_f32_against_f64(sc, cam, mask, planes)
    both = r["both"]
    assert both.sum() > 100
    # the decisions excused for lying within their bound of a boundary are few
    assert (both & ~r["margins"]["rect"]).sum() <= max(2, 0.01 * both.sum())
    # the bound is tight enough to mean something: the typical relative bound
    # of the exponent coefficients is a few hundred units in the last place,
    # so a slip that moves them by 1e-4 relative fails the pin
    for k in ("A2", "beta", "G2"):
        rel = r["bounds"][k][both] / np.maximum(np.abs(r["p64"][k][both]), 1e-12)
        assert np.median(rel) < 1e-4, (k, float(np.median(rel)))


def test_branch_scene_reaches_every_regime():
    sc, cam, planes, groups = branch_scene()
    p64 = oracle.preprocess(sc, cam, 0xFFFFFFFF, planes, "f64")
    W = cam.R.astype(np.float64)
    p = sc.means.astype(np.float64) @ W.T + cam.t.astype(np.float64)
    limx = 1.3 * 0.5 * cam.width / cam.fx
    limy = 1.3 * 0.5 * cam.height / cam.fy
    vis = p64["vis"] > 0
    for name, idx in groups.items():
        assert vis[idx].sum() >= max(3, len(idx) // 2), name
    g = groups["clamp"]
    clamped = (np.abs(p[g, 0] / p[g, 2]) > limx) | (np.abs(p[g, 1] / p[g, 2]) > limy)
    assert (clamped & vis[g]).sum() >= 10
    g = groups["clamp_edge"]
    assert (np.abs(np.abs(p[g, 0] / p[g, 2]) / limx - 1) < 2e-4).all()
    g = groups["near"]
    assert ((p[g, 2] - cam.znear < 1.1e-3) & vis[g]).sum() >= 10
    # the thin covariances project to (almost) rank-deficient 2x2 forms before the dilation
    cov = p64["cov2d"]
    for name in ("line", "point", "edge_on"):
        g = groups[name][vis[groups[name]]]
        pre_det = (cov[g, 0] - 0.3) * (cov[g, 2] - 0.3) - cov[g, 1] ** 2
        assert (np.abs(pre_det) < 1e-3 * np.maximum(1e-12, (cov[g, 0] - 0.3) * (cov[g, 2] - 0.3)) + 1e-20).any(), name
    g = groups["opaque"]
    assert (p64["rgb"][g] == 0).any() and (p64["opac"][g] > 1 - 1e-12).any()


# --------------------------------------------------------------------------- planted mistakes

# Each mistake is a plausible slip in the single-precision projection; the pin
# above must reject every one on the branch scene.  The text replaced is
# matched exactly once in the oracle source.
PLANTED = {
    "upper frustum clamp with the wrong sign": (
        "float cxz = fminf(limx, fmaxf(-limx, izx));",
        "float cxz = izx > limx ? -limx : fmaxf(-limx, izx);"),
    "frustum clamp limit 1.2 instead of 1.3": (
        "float limx = 1.3f * ((0.5f * (float)W) / fx);", "float limx = 1.2f * ((0.5f * (float)W) / fx);"),
    "dilation dropped from Sigma'_11": (
        "float c11 = ((u10 * t10 + u11 * t11) + u12 * t12) + 0.3f;",
        "float c11 = ((u10 * t10 + u11 * t11) + u12 * t12) + 0.0f;"),
    "beta with the wrong sign": ("beta[i] = -(c01 / c11);", "beta[i] = (c01 / c11);"),
    "quaternion not normalised": (
        "float w = qw / qnrm, x = qx / qnrm, y = qy / qnrm, z = qz / qnrm;",
        "float w = qw, x = qx, y = qy, z = qz;"),
    "camera rotation transposed in T": (
        "float t00 = j00 * Rc[0] + j02 * Rc[6], t01 = j00 * Rc[1] + j02 * Rc[7]",
        "float t00 = j00 * Rc[0] + j02 * Rc[6], t01 = j00 * Rc[3] + j02 * Rc[7]"),
    "clamped y offset taken from x": ("j12 = -(fy * cyz) / pz;", "j12 = -(fy * cxz) / pz;"),
    "scale squared once too often": ("float m00 = r00 * s0, m01 = r01 * s1, m02 = r02 * s2;",
                                     "float m00 = r00 * s0 * s0, m01 = r01 * s1, m02 = r02 * s2;"),
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_pin_rejects_planted_mistake(name, tmp_path):
    old, new = PLANTED[name]
    with open(oracle.source_path()) as f:
        src = f.read()
    assert src.count(old) == 1, "planted-mistake anchor not found: " + old
    sc, cam, planes, _ = branch_scene()
    with oracle.variant(src.replace(old, new), str(tmp_path)):
        with pytest.raises(AssertionError):
            check_f32_against_f64(sc, cam, 0xFFFFFFFF, planes)
    # and the unmodified oracle passes
    check_f32_against_f64(sc, cam, 0xFFFFFFFF, planes)


def test_f32_render_close_to_f64_render():
    w = synth.scene_c2(scale=0.005, width=128, height=128)
    sc, cam = w["scene"], w["cameras"][0]
    a = oracle.render(sc, cam, w["layer_mask"], w["planes"], w["bg"], "f64")
    b = oracle.render(sc, cam, w["layer_mask"], w["planes"], w["bg"], "f32")
    mse = ((a["image"] - b["image"]) ** 2).mean()
    assert mse == 0 or 10 * math.log10(1.0 / mse) > 80


def test_f32_half_storage_dequantises_exactly():
    w = synth.scene_c1(scale=0.1)
    sc = w["scene"]
    for kind in ("f16", "bf16"):
        q = synth.from_half_storage(synth.to_half_storage(sc.sh, kind), kind)
        # widening back is exact: re-quantising gives the same bits
        assert np.array_equal(synth.to_half_storage(q, kind), synth.to_half_storage(sc.sh, kind))
        rel = np.abs(q - sc.sh) / np.maximum(np.abs(sc.sh), 1e-3)
        assert rel.max() < (2 ** -10 if kind == "f16" else 2 ** -7)

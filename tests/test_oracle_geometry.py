"""Pins of the oracle's per-Gaussian projection (EWA splatting, Sec. 2.2.1 and
Sec. 3.3) against geometry computed independently of it."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from synth import look_at_camera
from tests.helpers import axis_camera, make_scene, random_small_scene


def test_quaternion_rotation_matches_scipy():
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        R = oracle.quat_to_rot(q)
        Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: (x, y, z, w)
        assert np.abs(R - Rs).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-13


def test_quarter_turn_about_z():
    c = math.cos(math.pi / 4)
    R = oracle.quat_to_rot([c, 0, 0, c])
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def _pinhole(cam, mu):
    p = cam.R.astype(np.float64) @ np.asarray(mu, np.float64) + cam.t.astype(np.float64)
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def test_mean_projects_like_a_pinhole():
    sc = random_small_scene(4, n=30)
    cam = look_at_camera((1.0, -0.5, 3.5), width=96, height=64)
    pre = oracle.preprocess(sc, cam)
    for i in np.nonzero(pre["vis"])[0]:
        uv = _pinhole(cam, sc.means[i])
        assert abs(pre["u"][i] - uv[0]) < 1e-9 and abs(pre["v"][i] - uv[1]) < 1e-9
    R = cam.R.astype(np.float64)
    assert np.allclose(pre["depth"][pre["vis"] > 0],
                       (sc.means.astype(np.float64) @ R.T + cam.t)[pre["vis"] > 0, 2], atol=1e-12)


def test_screen_covariance_is_jacobian_sandwich():
    # Sigma' - 0.3 I = J_pi Sigma J_pi^T with J_pi the derivative of the pinhole
    # projection at the mean (finite differences) and Sigma from scipy rotations.
    sc = random_small_scene(5, n=40, extent=0.3)
    cam = look_at_camera((0.4, 0.3, 3.0), width=128, height=128)
    pre = oracle.preprocess(sc, cam)
    h = 1e-6
    checked = 0
    for i in np.nonzero(pre["vis"])[0]:
        mu = sc.means[i].astype(np.float64)
        Jpi = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            Jpi[:, j] = (_pinhole(cam, mu + e) - _pinhole(cam, mu - e)) / (2 * h)
        q = sc.quats[i].astype(np.float64)
        q /= np.linalg.norm(q)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(np.exp(2 * sc.log_scales[i].astype(np.float64))) @ R.T
        S2 = Jpi @ Sig @ Jpi.T + 0.3 * np.eye(2)
        got = np.array([[pre["cov2d"][i, 0], pre["cov2d"][i, 1]], [pre["cov2d"][i, 1], pre["cov2d"][i, 2]]])
        assert np.abs(got - S2).max() < 1e-6 * max(1.0, np.abs(S2).max())
        # exponent coefficients reproduce -1/2 log2(e) d^T Sigma'^-1 d
        Q = np.linalg.inv(S2)
        rng = np.random.default_rng(i)
        for d in rng.normal(0, 3, (5, 2)):
            p = d[0] + pre["beta"][i] * d[1]
            e2 = pre["A2"][i] * p * p + pre["G2"][i] * d[1] * d[1]
            assert abs(e2 - (-0.5 / math.log(2)) * d @ Q @ d) < 1e-6 * max(1.0, abs(e2))
        checked += 1
    assert checked > 10


def test_isotropic_gaussian_on_axis_closed_form():
    z0, s = 4.0, 0.05
    cam = axis_camera(z0, 33, 33)
    sc = make_scene([[0, 0, 0]], math.log(s), rgb=[0.2, 0.4, 0.6], opacity_logit=0.5)
    pre = oracle.preprocess(sc, cam)
    s = math.exp(float(sc.log_scales[0, 0]))          # the stored (float32) log-scale
    sig2 = (cam.fx * s / z0) ** 2 + 0.3
    assert pre["vis"][0] == 1
    assert abs(pre["u"][0] - 16.5) < 1e-12 and abs(pre["v"][0] - 16.5) < 1e-12
    assert np.allclose(pre["cov2d"][0], [sig2, 0.0, sig2], rtol=1e-12, atol=1e-12)
    # mid^2 - det = 0, so lambda_max = sigma'^2 + sqrt(0.1)
    assert pre["radius"][0] == math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    assert abs(pre["beta"][0]) < 1e-15
    assert abs(pre["A2"][0] - (-0.5 / math.log(2)) / sig2) < 1e-12
    assert np.allclose(pre["rgb"][0], [0.2, 0.4, 0.6], atol=1e-7)   # SH DC stored in float32
    assert abs(pre["opac"][0] - 1 / (1 + math.exp(-0.5))) < 1e-15


def test_near_plane_cull():
    cam = axis_camera(4.0)
    # depth = 4 - z; znear = 0.2 keeps depth > 0.2 only
    sc = make_scene([[0, 0, 3.79], [0, 0, 3.81], [0, 0, 3.8 - 1e-4]], -3.0)
    pre = oracle.preprocess(sc, cam)
    assert list(pre["vis"]) == [1, 0, 1]


def test_layer_mask_and_planes_cull():
    cam = axis_camera(4.0, 64, 64)
    sc = make_scene([[0.1, 0, 0], [-0.1, 0, 0], [0.1, 0.05, 0], [-0.1, 0.05, 0]], -3.0,
                    layer=[0, 0, 1, 1])
    pre = oracle.preprocess(sc, cam, layer_mask=0b10)
    assert list(pre["vis"]) == [0, 0, 1, 1]
    plane = (np.array([1.0, 0.0, 0.0], np.float32), np.float32(0.0), 0b10)   # keep x >= 0 in layer 1
    pre = oracle.preprocess(sc, cam, layer_mask=0b11, planes=[plane])
    assert list(pre["vis"]) == [1, 1, 1, 0]
    plane_all = (np.array([1.0, 0.0, 0.0], np.float32), np.float32(0.0), 0xFFFFFFFF)
    pre = oracle.preprocess(sc, cam, layer_mask=0b11, planes=[plane_all])
    assert list(pre["vis"]) == [1, 0, 1, 0]


def test_offscreen_gaussian_has_empty_rect():
    cam = axis_camera(4.0, 32, 32)
    sc = make_scene([[3.0, 0, 0], [0, 0, 0]], -4.0)
    pre = oracle.preprocess(sc, cam)
    assert list(pre["vis"]) == [0, 1]


@pytest.mark.parametrize("seed", [6, 7])
def test_frustum_clamp_uses_boundary_jacobian(seed):
    # Outside 1.3x the half field of view the Jacobian is taken at the clamped
    # ray x/z = +-1.3 tan(fov/2): compare with the pinhole derivative there.
    cam = axis_camera(4.0, 64, 64)
    lim = 1.3 * 0.5 * cam.width / cam.fx
    rng = np.random.default_rng(seed)
    z = 2.0
    mu = np.array([lim * z * 1.2 + 0.0, rng.uniform(-0.1, 0.1), 4.0 - z])   # depth z, beyond the clamp in x
    sc = make_scene([mu], np.log([0.5, 0.4, 0.3]))
    pre = oracle.preprocess(sc, cam)
    if not pre["vis"][0]:
        pytest.skip("rect empty for this draw")
    W = cam.R.astype(np.float64)
    p = W @ sc.means[0].astype(np.float64) + cam.t.astype(np.float64)
    z = p[2]
    assert p[0] / z > lim
    pc = np.array([lim * z, p[1], z])
    J = np.array([[cam.fx / z, 0, -cam.fx * pc[0] / z ** 2], [0, cam.fy / z, -cam.fy * pc[1] / z ** 2]])
    Sig = np.diag(np.exp(2 * sc.log_scales[0].astype(np.float64)))
    S2 = J @ W @ Sig @ W.T @ J.T + 0.3 * np.eye(2)
    assert np.allclose(pre["cov2d"][0], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-9)

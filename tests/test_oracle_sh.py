"""Pins of the oracle's real spherical harmonics (view-dependent colour, Sec. 3.1:
specular effects approximated through SH; Sec. 3.3: SH are ~3/4 of the model)."""
import math

import numpy as np
import pytest

import oracle


def _dirs(rng, n):
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_orthonormal_by_exact_quadrature():
    # Gauss-Legendre in z (8 nodes) x uniform in phi (16 nodes) integrates every
    # product Y_i Y_j (degree <= 6) exactly, so the Gram matrix must be the identity.
    zs, wz = np.polynomial.legendre.leggauss(8)
    phis = 2 * math.pi * np.arange(16) / 16
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for ph in phis:
            Y = oracle.sh_basis(3, [s * math.cos(ph), s * math.sin(ph), z])
            G += np.outer(Y, Y) * w * (2 * math.pi / 16)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_addition_theorem():
    # sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every unit direction
    rng = np.random.default_rng(0)
    for d in _dirs(rng, 50):
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            s = sum(Y[l * l + l + m] ** 2 for m in range(-l, l + 1))
            assert abs(s - (2 * l + 1) / (4 * math.pi)) < 1e-13


def test_textbook_cartesian_forms():
    # Standard table of real SH with the Condon-Shortley phase, ordered m = -l..l.
    rng = np.random.default_rng(1)
    for x, y, z in _dirs(rng, 20):
        Y = oracle.sh_basis(3, [x, y, z])
        ref = [
            0.5 * math.sqrt(1 / math.pi),
            -math.sqrt(3 / (4 * math.pi)) * y,
            math.sqrt(3 / (4 * math.pi)) * z,
            -math.sqrt(3 / (4 * math.pi)) * x,
            0.5 * math.sqrt(15 / math.pi) * x * y,
            -0.5 * math.sqrt(15 / math.pi) * y * z,
            0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1),
            -0.5 * math.sqrt(15 / math.pi) * x * z,
            0.25 * math.sqrt(15 / math.pi) * (x * x - y * y),
            -0.25 * math.sqrt(35 / (2 * math.pi)) * y * (3 * x * x - y * y),
            0.5 * math.sqrt(105 / math.pi) * x * y * z,
            -0.25 * math.sqrt(21 / (2 * math.pi)) * y * (5 * z * z - 1),
            0.25 * math.sqrt(7 / math.pi) * z * (5 * z * z - 3),
            -0.25 * math.sqrt(21 / (2 * math.pi)) * x * (5 * z * z - 1),
            0.25 * math.sqrt(105 / math.pi) * z * (x * x - y * y),
            -0.25 * math.sqrt(35 / (2 * math.pi)) * x * (x * x - 3 * y * y),
        ]
        assert np.abs(Y - np.array(ref)).max() < 1e-13


def test_axis_values():
    # On +z only the m = 0 functions are non-zero: Y_l0 = sqrt((2l+1)/(4 pi)).
    Y = oracle.sh_basis(3, [0.0, 0.0, 1.0])
    for l in range(4):
        for m in range(-l, l + 1):
            want = math.sqrt((2 * l + 1) / (4 * math.pi)) if m == 0 else 0.0
            assert abs(Y[l * l + l + m] - want) < 1e-14


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_lower_degree_is_prefix(deg):
    d = [0.3, -0.5, 0.81]
    d = np.array(d) / np.linalg.norm(d)
    assert np.array_equal(oracle.sh_basis(deg, d), oracle.sh_basis(3, d)[: (deg + 1) ** 2])


def test_direction_derivative_finite_differences():
    rng = np.random.default_rng(2)
    h = 1e-6
    for d in _dirs(rng, 10):
        _, dY = oracle.sh_basis(3, d, grad=True)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            fd = (oracle.sh_basis(3, d + e) - oracle.sh_basis(3, d - e)) / (2 * h)
            assert np.abs(fd - dY[:, j]).max() < 1e-8

"""Pins of the SH-codebook oracle (K-means) against an independent library
evaluation, the per-cluster mean written as a loop, and exact recovery of
well-separated clusters."""
import numpy as np
import pytest

from oracle import codebook as CB


def test_assign_matches_scipy_cdist():
    sp = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((300, 45))
    c = rng.standard_normal((37, 45))
    ref = np.argmin(sp.cdist(x, c, "sqeuclidean"), axis=1)
    assert np.array_equal(CB.kmeans_assign(x, c), ref)


def test_update_is_the_cluster_mean():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((200, 9))
    c0 = rng.standard_normal((12, 9))
    a = rng.integers(0, 10, 200)          # clusters 10 and 11 stay empty
    c1 = CB.kmeans_update(x, a, c0)
    for j in range(12):
        members = [x[i] for i in range(200) if a[i] == j]
        want = np.mean(members, axis=0) if members else c0[j]
        assert np.allclose(c1[j], want, rtol=0, atol=1e-14)


def test_lloyd_recovers_separated_clusters():
    rng = np.random.default_rng(2)
    centers = rng.standard_normal((8, 6)) * 10
    lab = rng.integers(0, 8, 800)
    x = centers[lab] + rng.standard_normal((800, 6)) * 0.01
    c = x[[np.nonzero(lab == j)[0][0] for j in range(8)]]     # one seed point per cluster
    for _ in range(3):
        a = CB.kmeans_assign(x, c)
        c = CB.kmeans_update(x, a, c)
    assert np.array_equal(a, lab)
    assert np.abs(c - centers).max() < 5e-3
    assert CB.sq_dist(x, c, a).max() < 1e-2


def test_dequantise_definition():
    rng = np.random.default_rng(3)
    K = 4
    dc = rng.standard_normal((5, 3))
    cb = rng.standard_normal((3, 16)).astype(np.float16)     # rows padded past 3(K-1) = 9
    a = np.array([2, 0, 1, 2, 2])
    sh = CB.dequantise(dc, cb, a, K)
    assert np.array_equal(sh[:, 0], dc)
    for i in range(5):
        assert np.array_equal(sh[i, 1:].reshape(-1), cb[a[i], :9].astype(np.float64))

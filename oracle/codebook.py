"""FP64 oracle of the SH codebook (Sec. 3.3: SH coefficients, about 3/4 of a
model's size, are clustered with K-means across all layers; Sec. 4.3).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
oracle legs of ``bench.py`` may import this module.  Plain numpy in double
precision; no code is shared with ``paper_2410_16978_gb300``.

Definitions (Lloyd's K-means iteration):
* assign: a[i] = argmin_j |x_i - c_j|^2 (ties to the lower index);
* update: c_j = mean of the points assigned to j; a cluster with no point
  keeps its centroid;
* storage: the DC coefficient (k = 0) of every Gaussian stays per Gaussian;
  the rest (k >= 1, 3(K - 1) values) is replaced by its centroid, stored in
  FP16; dequantised SH = [DC, fp16(c_{a[i]})].

Parity status: assign pinned by scipy.spatial.distance.cdist and by exact
recovery of well-separated clusters; update pinned by the per-cluster mean
written as a loop; dequantisation pinned by its definition.
"""
from __future__ import annotations

import numpy as np


def kmeans_assign(points, centroids) -> np.ndarray:
    x = np.asarray(points, np.float64)
    c = np.asarray(centroids, np.float64)
    d = ((x[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    return np.argmin(d, axis=1)


def sq_dist(points, centroids, assign) -> np.ndarray:
    x = np.asarray(points, np.float64)
    c = np.asarray(centroids, np.float64)
    return ((x - c[np.asarray(assign)]) ** 2).sum(-1)


def kmeans_update(points, assign, centroids) -> np.ndarray:
    x = np.asarray(points, np.float64)
    c = np.array(centroids, np.float64)
    a = np.asarray(assign)
    sums = np.zeros_like(c)
    cnt = np.zeros(c.shape[0])
    np.add.at(sums, a, x)
    np.add.at(cnt, a, 1.0)
    nz = cnt > 0
    c[nz] = sums[nz] / cnt[nz, None]
    return c


def dequantise(dc, centroids_f16, assign, K: int) -> np.ndarray:
    """SH [N][K][3] from per-Gaussian DC [N][3] and FP16 centroids [C][>= 3(K-1)]."""
    n = np.asarray(dc).shape[0]
    out = np.zeros((n, K, 3))
    out[:, 0, :] = np.asarray(dc, np.float64)
    rest = np.asarray(centroids_f16)[np.asarray(assign), :3 * (K - 1)].astype(np.float64)
    out[:, 1:, :] = rest.reshape(n, K - 1, 3)
    return out

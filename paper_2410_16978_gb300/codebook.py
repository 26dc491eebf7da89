"""SH codebook of a layered model (Sec. 3.3: the SH coefficients, about 3/4
of the model, are clustered with K-means across all layers so that every
layer shares one palette; Sec. 4.3).  An offline step before rendering: Lloyd
iterations on the device (gs_kmeans_assign / gs_kmeans_update) over the
coefficients k >= 1 of every Gaussian, then gs_sh_codebook_encode writes the
per-Gaussian DC coefficient, a 16-bit index and the FP16 table.  The result
is a render-only DeviceScene with sh_dtype "cb".
"""
from __future__ import annotations

import torch

from . import _lib
from .api import DeviceScene, _stream_handle


def _ptr_offset(t: torch.Tensor, floats: int) -> int:
    return t.data_ptr() + 4 * floats


def build_sh_codebook(scene: DeviceScene, size: int = 16384, iters: int = 8, sample: int = 0, seed: int = 0,
                      stream=None):
    """Clusters the SH coefficients k >= 1 of a float32-SH scene into `size`
    centroids (Lloyd's iteration, `iters` rounds, seeded with distinct random
    Gaussians; with 0 < `sample` < N the rounds run on that many random
    Gaussians and every Gaussian is assigned at the end).  Returns
    (codebook scene, centroids float32 [k][3(K-1)], assignment uint32 [N]).
    The float32 scene is left untouched."""
    if scene.sh_dtype != "f32":
        raise ValueError("the codebook is built from float32 SH")
    if scene.sh_degree < 1:
        raise ValueError("SH degree 0 has nothing to cluster")
    if not 1 <= size <= 65536:
        raise ValueError("codebook size must be 1..65536")
    dev = scene.sh.device
    n = scene.n
    K = (scene.sh_degree + 1) ** 2
    row = 3 * K                       # floats per Gaussian in sh
    dim = 3 * (K - 1)                 # clustered coefficients, at offset 3 of every row
    st = _stream_handle(stream)
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    sh_flat = scene.sh.reshape(n, row)
    if 0 < sample < n:
        pick = torch.randperm(n, generator=gen)[:sample].to(torch.int32).to(dev)
        train = torch.empty((sample, row), dtype=torch.float32, device=dev)
        _lib.gs_gather_rows(sh_flat, train, row * 4, pick, sample, st)
        m = sample
    else:
        train, m = sh_flat, n
    k = min(size, m)
    # seeds: k distinct training rows; a k-means update of those rows with the
    # identity assignment makes every centroid exactly its seed
    seed_idx = torch.randperm(m, generator=gen)[:k].to(torch.int32).to(dev)
    seed_rows = torch.empty((k, row), dtype=torch.float32, device=dev)
    _lib.gs_gather_rows(train, seed_rows, row * 4, seed_idx, k, st)
    cent = torch.zeros((k, dim), dtype=torch.float32, device=dev)
    ident = torch.arange(k, dtype=torch.int32, device=dev)
    scratch_bytes = _lib.gs_kmeans_scratch_size(k, dim)
    scratch = torch.empty(scratch_bytes, dtype=torch.uint8, device=dev)
    _lib.gs_kmeans_update(_ptr_offset(seed_rows, 3), k, dim, row, ident, k, cent, scratch, scratch_bytes, st)
    assign_t = torch.empty(m, dtype=torch.int32, device=dev)
    for _ in range(int(iters)):
        _lib.gs_kmeans_assign(_ptr_offset(train, 3), m, dim, row, cent, k, assign_t, st)
        _lib.gs_kmeans_update(_ptr_offset(train, 3), m, dim, row, assign_t, k, cent, scratch, scratch_bytes, st)
    assign = torch.empty(n, dtype=torch.int32, device=dev)
    _lib.gs_kmeans_assign(_ptr_offset(sh_flat, 3), n, dim, row, cent, k, assign, st)
    rows_h = (dim + 7) // 8 * 8
    dc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    index = torch.empty(n, dtype=torch.int16, device=dev)       # bit pattern of uint16
    table = torch.empty((k, rows_h), dtype=torch.float16, device=dev)
    _lib.gs_sh_codebook_encode(scene.sh, n, scene.sh_degree, assign, cent, k, dc, index, table, st)
    cb = DeviceScene(scene.means, scene.log_scales, scene.quats, scene.opacity_logit, dc, scene.layer,
                     scene.sh_degree, "cb", scene.sr_dtype, sh_index=index, sh_table=table)
    return cb, cent, assign

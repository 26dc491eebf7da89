"""Layered Gaussian-splatting tile rasterizer for GB300 (sm_103a).

Hot path (all in hand-written CUDA in csrc/, behind the C ABI of include/gs.h):
per-Gaussian EWA projection with SH colour, tile binning after a depth-keyed
radix sort, front-to-back compositing honouring layer masks and clip planes,
and the backward pass with per-Gaussian contribution accumulation and prune.
"""
from ._lib import (  # noqa: F401
    GsError,
    gs_contrib_prune,
    gs_kernel_launches,
    gs_profile_collect,
    gs_profile_enable,
    gs_last_error_string,
    gs_prune_workspace_size,
    gs_read_status,
    gs_render,
    gs_render_backward,
    gs_render_batch,
    gs_render_workspace_size,
    gs_version,
    gs_workspace_layout,
    make_camera,
)
from .api import DeviceScene, Rasterizer, RenderFunction, contrib_prune, render  # noqa: F401
from .checkpoint import load_ply, load_scene, load_trainer, merge_layers, save_ply, save_scene, save_trainer  # noqa: F401

__version__ = "0.2.0"

"""The C ABI library loads, exports every entry point include/gs.h declares,
and rejects bad arguments on the host before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2410_16978_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gs_render", "gs_render_backward", "gs_contrib_prune"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    for name in _declared():
        assert hasattr(L, name), name
        assert name in _lib.EXPORTED, name


def test_version_and_empty_error():
    assert "sm_103a" in _lib.gs_version()


def test_settings_are_the_methods_constants():
    s = _lib.gs_get_settings()
    f32 = lambda x: float(ctypes.c_float(x).value)
    assert s.tile == 16 and s.checkpoint_stride == 256 and s.max_sh_degree == 3
    assert s.dilation == f32(0.3) and s.alpha_max == f32(0.99) and s.t_min == f32(1e-4)
    assert s.alpha_min == f32(1.0 / 255.0) and s.frustum_clamp == f32(1.3)
    assert s.radius_sigmas == 3.0 and s.eigen_floor == f32(0.1)
    assert (s.max_planes, s.max_image_dim, s.max_batch) == (_lib.GS_MAX_PLANES, 4096, _lib.GS_MAX_BATCH)
    assert s.debug_build == 0


def test_debug_library_exports_the_same_boundary():
    """libgs_debug.so (GS_DEBUG) has every entry point, says it is the debug
    build, and its hooks are refused by the release library."""
    D = _lib.load_debug()
    for name in _declared():
        assert hasattr(D, name), name
    assert D.gs_debug_build() == 1 and _lib.load().gs_debug_build() == 0
    with _lib.use(D):
        assert _lib.gs_get_settings().debug_build == 1
        _lib.gs_debug_sort_wait(0, -1)                  # host-only: resets the hook
        with pytest.raises(_lib.GsError) as e:
            _lib.gs_debug_sort_wait(100, 0)             # the first digit kernel has no wait
        assert e.value.code == _lib.GS_ERR_INVALID
    for call in (lambda: _lib.gs_debug_sort_wait(100, 1), lambda: _lib.gs_debug_site(None, 0)):
        with pytest.raises(_lib.GsError) as e:
            call()
        assert e.value.code == _lib.GS_ERR_INVALID


def test_workspace_size_and_layout():
    b = _lib.gs_render_workspace_size(1000, 100, 70, 5000)
    lay = _lib.gs_workspace_layout(1000, 100, 70, b)
    assert lay["total"] <= b and lay["dup_capacity"] >= 5000 - 64
    offs = [lay[k] for k in _lib.LAYOUT_NAMES[:9]]     # the regions (total and capacity follow)
    assert all(o % 256 == 0 for o in offs)
    assert len(set(offs)) == len(offs)
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_render_workspace_size(-1, 100, 70, 10)
    assert e.value.code == _lib.GS_ERR_INVALID
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_render_workspace_size(10, 0, 70, 10)
    assert e.value.code == _lib.GS_ERR_INVALID
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_workspace_layout(1000, 100, 70, 1024)
    assert e.value.code == _lib.GS_ERR_WORKSPACE
    _lib.gs_render_workspace_size(10, 4096, 4096, 10)          # the largest image
    for w, h in ((4097, 16), (16, 4097)):
        with pytest.raises(_lib.GsError) as e:
            _lib.gs_render_workspace_size(10, w, h, 10)
        assert e.value.code == _lib.GS_ERR_INVALID


def test_workspace_size_grows_with_the_scene():
    # a workspace sized for n Gaussians holds any smaller scene: the size never
    # drops as n grows, also where the depth sort's tile count (4096 Gaussians a
    # tile) crosses the squares at which its group size doubles
    for tiles in (1, 4, 16, 256, 1024, 4096, 16384, 65536):
        prev = 0
        for n in range(max(0, 4096 * tiles - 3), 4096 * tiles + 4):
            b = _lib.gs_render_workspace_size(n, 1024, 1024, 1_000_000)
            assert b >= prev, (n, b, prev)
            prev = b
    sizes = [_lib.gs_render_workspace_size(n, 512, 512, 100_000) for n in range(0, 3_000_000, 65_537)]
    assert sizes == sorted(sizes)


@pytest.mark.parametrize("W,H,n", [(1024, 1024, 1_200_000), (2064, 2208, 3_000_000)])
def test_workspace_size_grows_with_the_pair_capacity(W, H, n):
    # the workspace must grow with the pair capacity, so that a workspace
    # sized for C pairs holds at least C (checked across the capacities where
    # pieces of 128 k entries would outgrow a 64 MiB count matrix, the points
    # where an earlier sizing rule doubled the pieces)
    Tx = (W + 15) // 16
    for k in (1, 2, 4):
        t = k * ((1 << 31) // Tx)           # where pieces of 128 k entries would outgrow the budget
        prev = 0
        for c in range(t - 600, t + 600, 23):
            b = _lib.gs_render_workspace_size(n, W, H, c)
            assert b >= prev, (c, b, prev)
            prev = b
            if c % 5 == 0:
                assert _lib.gs_workspace_layout(n, W, H, b)["dup_capacity"] >= c, c


def test_render_rejects_bad_arguments_on_host():
    L = _lib.load()
    cam = _lib.gs_camera()
    cam.width, cam.height, cam.fx, cam.fy = 64, 64, 50.0, 50.0
    sc = _lib.gs_scene()
    sc.n = 10
    bg = (ctypes.c_float * 3)(0, 0, 0)
    rc = L.gs_render(None, ctypes.byref(cam), 1, None, 0, bg, None, 0, None, None, None)
    assert rc == _lib.GS_ERR_INVALID and "scene" in _lib.gs_last_error_string()
    rc = L.gs_render(ctypes.byref(sc), ctypes.byref(cam), 1, None, 0, bg, None, 0, None, None, None)
    assert rc == _lib.GS_ERR_INVALID                     # NULL scene arrays
    sc.n, sc.sh_degree = 0, 4
    rc = L.gs_render(ctypes.byref(sc), ctypes.byref(cam), 1, None, 0, bg, None, 0, None, None, None)
    assert rc == _lib.GS_ERR_INVALID and "sh_degree" in _lib.gs_last_error_string()
    sc.sh_degree = 0
    rc = L.gs_render(ctypes.byref(sc), ctypes.byref(cam), 1, None, 9, bg, None, 0, None, None, None)
    assert rc == _lib.GS_ERR_INVALID and "n_planes" in _lib.gs_last_error_string()
    cam.fx = 0.0
    rc = L.gs_render(ctypes.byref(sc), ctypes.byref(cam), 1, None, 0, bg, None, 0, None, None, None)
    assert rc == _lib.GS_ERR_INVALID


def test_prune_rejects_bad_arguments_on_host():
    L = _lib.load()
    assert L.gs_contrib_prune(None, 10, 0.005, None, None, None, None, 0, None) == _lib.GS_ERR_INVALID
    assert L.gs_contrib_prune(None, -1, 0.005, None, None, None, None, 0, None) == _lib.GS_ERR_INVALID
    n_keep = ctypes.c_int64()
    rc = L.gs_contrib_prune(None, 0, 0.005, None, None, ctypes.byref(n_keep), None, 0, None)
    assert rc == _lib.GS_ERR_WORKSPACE

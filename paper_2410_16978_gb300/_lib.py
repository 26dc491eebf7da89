"""ctypes binding of the C ABI in include/gs.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Pointers are
passed as integers (``tensor.data_ptr()``); host structs are built from plain
Python values.  No computation happens in this module: if the shared library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_P = ctypes.c_void_p

GS_OK, GS_ERR_INVALID, GS_ERR_WORKSPACE, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_OOM, GS_ERR_BOUNDS = range(7)
GS_DTYPE_SH_CODEBOOK = 3
GS_DTYPE_F32, GS_DTYPE_F16, GS_DTYPE_BF16 = 0, 1, 2
GS_TILE = 16
GS_MAX_PLANES = 8
GS_MAX_BATCH = 16

EXPORTED = ("gs_render_workspace_size", "gs_render", "gs_render_batch", "gs_render_stereo", "gs_render_backward", "gs_prune_workspace_size",
            "gs_contrib_prune", "gs_contrib_prune_noalloc", "gs_image_loss_workspace_size", "gs_image_loss",
            "gs_adam_step", "gs_activity_accumulate", "gs_activity_prune", "gs_gather_rows", "gs_kmeans_scratch_size",
            "gs_kmeans_assign", "gs_kmeans_update", "gs_sh_codebook_encode", "gs_workspace_layout", "gs_read_status", "gs_profile_enable",
            "gs_profile_collect", "gs_kernel_launches", "gs_get_settings", "gs_debug_build", "gs_debug_site",
            "gs_debug_sort_wait", "gs_last_error_string", "gs_version")
STAGES = ("preprocess", "compact", "depth_sort", "bin_rows", "bin_tiles", "composite_setup", "composite",
          "composite_bwd", "preprocess_bwd", "prune", "loss", "adam")
GS_LAYOUT_COUNT = 11
LAYOUT_NAMES = ("ctl", "rec", "tiles", "depth", "list", "ranges", "t_final", "n_contrib", "rec_grad", "total",
                "dup_capacity")


class gs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("znear", ctypes.c_float),
                ("_reserved", ctypes.c_float)]


class gs_clip_plane(ctypes.Structure):
    _fields_ = [("n", ctypes.c_float * 3), ("d", ctypes.c_float), ("layer_bits", ctypes.c_uint32),
                ("_reserved", ctypes.c_uint32)]


class gs_scene(ctypes.Structure):
    _fields_ = [("means", _P), ("log_scales", _P), ("quats", _P), ("opacity_logit", _P), ("sh", _P),
                ("layer", _P), ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("dtype_sh", ctypes.c_int32), ("dtype_scale_rot", ctypes.c_int32), ("sh_table_rows", ctypes.c_int32),
                ("sh_index", _P), ("sh_table", _P)]


class gs_grads(ctypes.Structure):
    _fields_ = [("means", _P), ("log_scales", _P), ("quats", _P), ("opacity_logit", _P), ("sh", _P)]


class gs_render_request(ctypes.Structure):
    _fields_ = [("scene", ctypes.POINTER(gs_scene)), ("camera", ctypes.POINTER(gs_camera)),
                ("layer_mask", ctypes.c_uint32), ("n_planes", ctypes.c_int32),
                ("planes", ctypes.POINTER(gs_clip_plane)), ("bg", ctypes.c_float * 3), ("_reserved", ctypes.c_float),
                ("workspace", _P), ("ws_bytes", ctypes.c_size_t), ("image", _P), ("alpha", _P)]


class gs_adam_state(ctypes.Structure):
    _fields_ = [("m", _P * 5), ("v", _P * 5)]


class gs_status(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("n_visible", ctypes.c_uint32), ("n_dup", ctypes.c_uint64),
                ("dup_capacity", ctypes.c_uint64), ("n_blended", ctypes.c_uint64)]


class gs_settings(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("dilation", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("t_min", ctypes.c_float), ("frustum_clamp", ctypes.c_float),
                ("radius_sigmas", ctypes.c_float), ("eigen_floor", ctypes.c_float),
                ("checkpoint_stride", ctypes.c_int32), ("max_sh_degree", ctypes.c_int32),
                ("max_planes", ctypes.c_int32), ("max_image_dim", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("debug_build", ctypes.c_int32)]


class GsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gs error %d: %s" % (code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libgs.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and (not os.path.exists(path) or _build._stale()):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("CUDA rasterizer library not built: %s" % path)
        _lib = _declare(ctypes.CDLL(path))
        return _lib


_debug_lib = None


def load_debug(build_if_missing: bool = True):
    """Loads libgs_debug.so, the GS_DEBUG build (bounds checks that report
    GS_ERR_BOUNDS through the status word, and the sort-wait test hook).  It is
    a separate library; ``use(load_debug())`` routes this module's calls to it."""
    global _debug_lib
    with _lock:
        if _debug_lib is None:
            path = _build.DEBUG_LIB
            if build_if_missing and (not os.path.exists(path) or _build._stale(path)):
                _build.build(debug=True)
            if not os.path.exists(path):
                raise RuntimeError("GS_DEBUG library not built: %s" % path)
            _debug_lib = _declare(ctypes.CDLL(path))
        return _debug_lib


class use:
    """``with _lib.use(lib):`` makes every function of this module call `lib`
    (e.g. the GS_DEBUG build) until the block ends."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _lib
        self.saved = load()
        _lib = self.lib
        return self.lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _declare(L):
    L.gs_render_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_size_t)]
    L.gs_render.argtypes = [ctypes.POINTER(gs_scene), ctypes.POINTER(gs_camera), ctypes.c_uint32,
                            ctypes.POINTER(gs_clip_plane), ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                            _P, ctypes.c_size_t, _P, _P, _P]
    L.gs_render_batch.argtypes = [ctypes.POINTER(gs_render_request), ctypes.c_int32, _P]
    L.gs_render_stereo.argtypes = [ctypes.POINTER(gs_scene), ctypes.POINTER(gs_camera), ctypes.POINTER(gs_camera),
                                   ctypes.c_uint32, ctypes.POINTER(gs_clip_plane), ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_float), _P, ctypes.c_size_t, _P, ctypes.c_size_t, _P,
                                   _P, _P, _P, ctypes.c_int32, _P]
    L.gs_render_backward.argtypes = [ctypes.POINTER(gs_scene), ctypes.POINTER(gs_camera),
                                     ctypes.POINTER(ctypes.c_float), _P, ctypes.c_size_t, _P, _P,
                                     ctypes.c_uint32, ctypes.POINTER(gs_grads), _P, _P, _P]
    L.gs_prune_workspace_size.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    L.gs_contrib_prune.argtypes = [_P, ctypes.c_int64, ctypes.c_float, _P, _P, _P, _P, ctypes.c_size_t, _P]
    L.gs_read_status.argtypes = [_P, ctypes.POINTER(gs_status), _P]
    L.gs_contrib_prune_noalloc.argtypes = [_P, ctypes.c_int64, ctypes.c_float, _P, _P, _P, _P]
    L.gs_image_loss_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
    L.gs_image_loss.argtypes = [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_float, ctypes.c_float, _P, ctypes.c_size_t, _P, _P, _P, _P]
    L.gs_adam_step.argtypes = [ctypes.POINTER(gs_scene), ctypes.POINTER(gs_grads), ctypes.POINTER(gs_adam_state),
                               ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_int32, ctypes.c_uint32, _P]
    L.gs_gather_rows.argtypes = [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P]
    L.gs_kmeans_scratch_size.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
    L.gs_kmeans_assign.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P, ctypes.c_int32, _P, _P]
    L.gs_kmeans_update.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P, ctypes.c_int32, _P, _P,
                                   ctypes.c_size_t, _P]
    L.gs_sh_codebook_encode.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, _P, _P]
    L.gs_activity_accumulate.argtypes = [ctypes.POINTER(gs_adam_state), _P, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_int32, ctypes.c_uint32, _P, _P]
    L.gs_activity_prune.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float, ctypes.c_float, _P,
                                    _P, _P, _P, ctypes.c_size_t, _P]
    L.gs_workspace_layout.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_int64)]
    L.gs_profile_enable.argtypes = [ctypes.c_int]
    L.gs_profile_collect.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.gs_kernel_launches.argtypes = []
    L.gs_last_error_string.restype = ctypes.c_char_p
    L.gs_version.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("gs_last_error_string", "gs_version"):
            getattr(L, name).restype = ctypes.c_int
    L.gs_kernel_launches.restype = ctypes.c_int64
    L.gs_get_settings.argtypes = [ctypes.POINTER(gs_settings)]
    L.gs_debug_build.argtypes = []
    L.gs_debug_site.argtypes = [_P, ctypes.POINTER(ctypes.c_uint32), _P]
    L.gs_debug_sort_wait.argtypes = [ctypes.c_uint32, ctypes.c_int32]
    return L


def _check(rc: int):
    if rc != GS_OK:
        raise GsError(rc, load().gs_last_error_string().decode())


# --------------------------------------------------------------------------- marshalling helpers

def make_camera(cam) -> gs_camera:
    """gs_camera from any object with R, t, fx, fy, cx, cy, width, height, znear."""
    c = gs_camera()
    R = [float(v) for row in cam.R for v in row] if hasattr(cam.R, "__len__") and len(cam.R) == 3 else \
        [float(v) for v in cam.R]
    for k in range(9):
        c.R[k] = R[k]
    for k in range(3):
        c.t[k] = float(cam.t[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(getattr(cam, "znear", 0.2))
    return c


def make_planes(planes):
    n = len(planes)
    if n > GS_MAX_PLANES:
        raise ValueError("at most %d clip planes" % GS_MAX_PLANES)
    arr = (gs_clip_plane * max(n, 1))()
    for k, (nrm, d, bits) in enumerate(planes):
        for j in range(3):
            arr[k].n[j] = float(nrm[j])
        arr[k].d = float(d)
        arr[k].layer_bits = int(bits) & 0xFFFFFFFF
    return arr, n


def _ptr(t):
    return None if t is None else ctypes.c_void_p(int(t) if isinstance(t, int) else t.data_ptr())


# --------------------------------------------------------------------------- the C entry points

def gs_render_workspace_size(n: int, width: int, height: int, dup_capacity: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().gs_render_workspace_size(int(n), int(width), int(height), int(dup_capacity), ctypes.byref(out)))
    return int(out.value)


def gs_render(scene: gs_scene, camera: gs_camera, layer_mask: int, planes, bg, workspace, ws_bytes: int, image,
              alpha, stream: int) -> None:
    parr, npl = make_planes(planes)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    _check(load().gs_render(ctypes.byref(scene), ctypes.byref(camera), int(layer_mask) & 0xFFFFFFFF, parr, npl, bgv,
                            _ptr(workspace), int(ws_bytes), _ptr(image), _ptr(alpha), ctypes.c_void_p(stream)))


def gs_render_batch(views, stream: int) -> None:
    """views: sequence of dicts with scene (gs_scene), camera (gs_camera), layer_mask, planes, bg,
    workspace, ws_bytes, image, alpha (alpha may be None)."""
    n = len(views)
    if not 1 <= n <= GS_MAX_BATCH:
        raise ValueError("1..%d views per batch" % GS_MAX_BATCH)
    reqs = (gs_render_request * n)()
    keep = []
    for k, v in enumerate(views):
        parr, npl = make_planes(v.get("planes", ()))
        keep.append((v["scene"], v["camera"], parr))
        reqs[k].scene = ctypes.pointer(v["scene"])
        reqs[k].camera = ctypes.pointer(v["camera"])
        reqs[k].layer_mask = int(v.get("layer_mask", 0xFFFFFFFF)) & 0xFFFFFFFF
        reqs[k].n_planes = npl
        reqs[k].planes = ctypes.cast(parr, ctypes.POINTER(gs_clip_plane))
        for j, b in enumerate(v.get("bg", (0.0, 0.0, 0.0))):
            reqs[k].bg[j] = float(b)
        reqs[k].workspace = _ptr(v["workspace"])
        reqs[k].ws_bytes = int(v["ws_bytes"])
        reqs[k].image = _ptr(v["image"])
        reqs[k].alpha = _ptr(v.get("alpha"))
    _check(load().gs_render_batch(reqs, n, ctypes.c_void_p(stream)))
    del keep


def gs_render_stereo(scene: gs_scene, left: gs_camera, right: gs_camera, layer_mask: int, planes, bg, ws_left,
                     ws_left_bytes: int, ws_right, ws_right_bytes: int, image_left, alpha_left, image_right,
                     alpha_right, shared_sort: bool, stream: int) -> None:
    parr, npl = make_planes(planes)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    _check(load().gs_render_stereo(ctypes.byref(scene), ctypes.byref(left), ctypes.byref(right),
                                   int(layer_mask) & 0xFFFFFFFF, parr, npl, bgv, _ptr(ws_left), int(ws_left_bytes),
                                   _ptr(ws_right), int(ws_right_bytes), _ptr(image_left), _ptr(alpha_left),
                                   _ptr(image_right), _ptr(alpha_right), 1 if shared_sort else 0,
                                   ctypes.c_void_p(stream)))


def gs_render_backward(scene: gs_scene, camera: gs_camera, bg, workspace, ws_bytes: int, dL_dimage, dL_dalpha,
                       grad_layer_mask: int, grads: gs_grads, contrib_sum, contrib_max, stream: int) -> None:
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    _check(load().gs_render_backward(ctypes.byref(scene), ctypes.byref(camera), bgv, _ptr(workspace), int(ws_bytes),
                                     _ptr(dL_dimage), _ptr(dL_dalpha), int(grad_layer_mask) & 0xFFFFFFFF,
                                     ctypes.byref(grads), _ptr(contrib_sum), _ptr(contrib_max),
                                     ctypes.c_void_p(stream)))


def gs_prune_workspace_size(n: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().gs_prune_workspace_size(int(n), ctypes.byref(out)))
    return int(out.value)


def gs_contrib_prune(contrib_max, n: int, threshold: float, keep, keep_index, n_keep, workspace, ws_bytes: int,
                     stream: int) -> None:
    _check(load().gs_contrib_prune(_ptr(contrib_max), int(n), float(threshold), _ptr(keep), _ptr(keep_index),
                                   _ptr(n_keep), _ptr(workspace), int(ws_bytes), ctypes.c_void_p(stream)))


def gs_contrib_prune_noalloc(contrib_max, n: int, threshold: float, keep, keep_index, n_keep, stream: int) -> None:
    _check(load().gs_contrib_prune_noalloc(_ptr(contrib_max), int(n), float(threshold), _ptr(keep), _ptr(keep_index),
                                           _ptr(n_keep), ctypes.c_void_p(stream)))


def gs_image_loss_workspace_size(width: int, height: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().gs_image_loss_workspace_size(int(width), int(height), ctypes.byref(out)))
    return int(out.value)


def gs_image_loss(image, alpha, target_rgb, target_alpha, bg, width: int, height: int, lambda_dssim: float,
                  w_alpha: float, workspace, ws_bytes: int, loss, dL_dimage, dL_dalpha, stream: int) -> None:
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    _check(load().gs_image_loss(_ptr(image), _ptr(alpha), _ptr(target_rgb), _ptr(target_alpha), bgv, int(width),
                                int(height), float(lambda_dssim), float(w_alpha), _ptr(workspace), int(ws_bytes),
                                _ptr(loss), _ptr(dL_dimage), _ptr(dL_dalpha), ctypes.c_void_p(stream)))


def gs_adam_step(scene: gs_scene, grads: gs_grads, state: gs_adam_state, lr, beta1: float, beta2: float, eps: float,
                 step: int, train_layer_mask: int, stream: int) -> None:
    lrv = (ctypes.c_float * 5)(*[float(v) for v in lr])
    _check(load().gs_adam_step(ctypes.byref(scene), ctypes.byref(grads), ctypes.byref(state), lrv, float(beta1),
                               float(beta2), float(eps), int(step), int(train_layer_mask) & 0xFFFFFFFF,
                               ctypes.c_void_p(stream)))


def gs_activity_accumulate(state: gs_adam_state, layer, n: int, sh_degree: int, lr, beta1: float, beta2: float,
                           eps: float, step: int, train_layer_mask: int, activity, stream: int) -> None:
    lrv = (ctypes.c_float * 5)(*[float(v) for v in lr])
    _check(load().gs_activity_accumulate(ctypes.byref(state), _ptr(layer), int(n), int(sh_degree), lrv, float(beta1),
                                         float(beta2), float(eps), int(step), int(train_layer_mask) & 0xFFFFFFFF,
                                         _ptr(activity), ctypes.c_void_p(stream)))


def gs_activity_prune(activity, layer, n: int, train_layer_mask: int, samples: float, threshold: float, keep,
                      keep_index, n_keep, workspace, ws_bytes: int, stream: int) -> None:
    _check(load().gs_activity_prune(_ptr(activity), _ptr(layer), int(n), int(train_layer_mask) & 0xFFFFFFFF,
                                    float(samples), float(threshold), _ptr(keep), _ptr(keep_index), _ptr(n_keep),
                                    _ptr(workspace), int(ws_bytes), ctypes.c_void_p(stream)))


def gs_kmeans_scratch_size(k: int, dim: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().gs_kmeans_scratch_size(int(k), int(dim), ctypes.byref(out)))
    return int(out.value)


def gs_kmeans_assign(points, n: int, dim: int, stride: int, centroids, k: int, assign, stream: int) -> None:
    _check(load().gs_kmeans_assign(_ptr(points), int(n), int(dim), int(stride), _ptr(centroids), int(k), _ptr(assign),
                                   ctypes.c_void_p(stream)))


def gs_kmeans_update(points, n: int, dim: int, stride: int, assign, k: int, centroids, scratch, scratch_bytes: int,
                     stream: int) -> None:
    _check(load().gs_kmeans_update(_ptr(points), int(n), int(dim), int(stride), _ptr(assign), int(k),
                                   _ptr(centroids), _ptr(scratch), int(scratch_bytes), ctypes.c_void_p(stream)))


def gs_sh_codebook_encode(sh, n: int, sh_degree: int, assign, centroids, k: int, dc, index, table,
                          stream: int) -> None:
    _check(load().gs_sh_codebook_encode(_ptr(sh), int(n), int(sh_degree), _ptr(assign), _ptr(centroids), int(k),
                                        _ptr(dc), _ptr(index), _ptr(table), ctypes.c_void_p(stream)))


def gs_gather_rows(src, dst, row_bytes: int, index, n: int, stream: int) -> None:
    _check(load().gs_gather_rows(_ptr(src), _ptr(dst), int(row_bytes), _ptr(index), int(n), ctypes.c_void_p(stream)))


def gs_workspace_layout(n: int, width: int, height: int, ws_bytes: int) -> dict:
    out = (ctypes.c_int64 * GS_LAYOUT_COUNT)()
    _check(load().gs_workspace_layout(int(n), int(width), int(height), int(ws_bytes), out))
    return dict(zip(LAYOUT_NAMES, [int(v) for v in out]))


def gs_read_status(workspace, stream: int) -> gs_status:
    st = gs_status()
    _check(load().gs_read_status(_ptr(workspace), ctypes.byref(st), ctypes.c_void_p(stream)))
    return st


def gs_profile_enable(on: bool) -> None:
    _check(load().gs_profile_enable(1 if on else 0))


def gs_profile_collect() -> dict:
    """{stage: (milliseconds, calls)} since the previous collect (waits for the events)."""
    ms = (ctypes.c_double * len(STAGES))()
    calls = (ctypes.c_int64 * len(STAGES))()
    _check(load().gs_profile_collect(ms, calls))
    return {name: (float(ms[k]), int(calls[k])) for k, name in enumerate(STAGES)}


def gs_kernel_launches() -> int:
    return int(load().gs_kernel_launches())


def gs_last_error_string() -> str:
    return load().gs_last_error_string().decode()


def gs_version() -> str:
    return load().gs_version().decode()


def gs_get_settings() -> gs_settings:
    out = gs_settings()
    _check(load().gs_get_settings(ctypes.byref(out)))
    return out


def gs_debug_build() -> bool:
    return bool(load().gs_debug_build())


def gs_debug_site(workspace, stream: int) -> int:
    out = ctypes.c_uint32(0)
    _check(load().gs_debug_site(_ptr(workspace), ctypes.byref(out), ctypes.c_void_p(stream)))
    return int(out.value)


def gs_debug_sort_wait(spin_limit: int, withhold_pass: int) -> None:
    _check(load().gs_debug_sort_wait(int(spin_limit), int(withhold_pass)))

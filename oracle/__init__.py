"""FP64 CPU oracle of the layered Gaussian-splatting rasterizer.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with ``paper_2410_16978_gb300`` and never calls it.

The arithmetic lives in ``gs_oracle.c`` (plain C, double precision, built with
gcc and ``-ffp-contract=off``); this module only builds it and marshals numpy
arrays.  See the header of ``gs_oracle.c`` for the equations and the paper
sections they follow.

Parity status of each function (what pins it in ``tests/test_oracle_*.py``):
  preprocess(f64)   closed forms (isotropic splat, covariance eigenvalues,
                    quaternion rotations, finite-difference Jacobian of the
                    perspective map), brute-force projection of samples
  preprocess(f32)   agreement with the f64 path within single-precision error;
                    integer decisions equal except at flagged boundaries
  sh_basis          Monte-Carlo orthonormality, addition theorem, textbook
                    closed forms, axis values
  bin_tiles         brute-force per-pixel render over all Gaussians; sorted
                    order checked against numpy lexsort
  composite         single-splat closed form, two-splat ordering, the
                    transmittance invariant, early-stop count, thresholds,
                    layer/clip equivalences, brute force
  composite_backward / chain
                    central finite differences of the forward
  prune             definition (threshold compare) on hand-made inputs
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compile gs_oracle.c with gcc (plain C99, no contraction of a*b+c)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def source_path() -> str:
    """Path of the oracle's C source (read by the planted-mistake tests)."""
    return _SRC


class variant:
    """``with oracle.variant(source_text, directory):`` builds a modified copy
    of the oracle's C source in ``directory`` and makes every function of this
    module use it until the block ends.  Only the planted-mistake tests use it:
    they check that the pins reject a deliberately wrong oracle."""

    def __init__(self, source_text: str, directory: str):
        self.src = os.path.join(directory, "gs_oracle_variant.c")
        self.so = os.path.join(directory, "liboracle_variant.so")
        with open(self.src, "w") as f:
            f.write(source_text)

    def __enter__(self):
        global _lib
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               self.src, "-o", self.so, "-lm"])
        self._saved = _load()
        _lib = _declare(ctypes.CDLL(self.so))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U32 = ctypes.c_uint32


def _load():
    global _lib
    if _lib is not None:
        return _lib
    _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    L.or_sh_basis.argtypes = [ctypes.c_int, _P, _P, _P]
    L.or_quat_to_rot.argtypes = [_P, _P]
    L.or_preprocess64.argtypes = ([_I64] + [_P] * 6 + [ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                  _U32, _P, _P, ctypes.c_int] + [_P] * 12)
    L.or_preprocess32.argtypes = ([_I64] + [_P] * 6 + [ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                  _U32, _P, _P, ctypes.c_int] + [_P] * 11)
    L.or_expf32.argtypes = [ctypes.c_float]
    L.or_expf32.restype = ctypes.c_float
    L.or_count_dups.argtypes = [_I64, _P, _P]
    L.or_count_dups.restype = _I64
    L.or_bin.argtypes = [_I64, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P]
    L.or_composite.argtypes = [ctypes.c_int, ctypes.c_int] + [_P] * 19
    L.or_composite_bruteforce.argtypes = [ctypes.c_int, ctypes.c_int, _I64, _P, _I64] + [_P] * 9
    L.or_composite_backward.argtypes = [ctypes.c_int, ctypes.c_int, _I64] + [_P] * 18
    L.or_composite_pixels.argtypes = [ctypes.c_int, ctypes.c_int] + [_P] * 10 + [_I64] + [_P] * 9
    L.or_chain.argtypes = ([_I64] + [_P] * 6 + [ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P, _P,
                           _U32] + [_P] * 5)
    L.or_prune.argtypes = [_I64, _P, ctypes.c_double, _P]
    L.or_prune.restype = _I64
    return L


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def cam_array(cam, dtype=np.float64) -> np.ndarray:
    """Flat camera: R (9, row-major world->camera), t (3), fx, fy, cx, cy, znear."""
    a = np.zeros(17, np.float32)
    a[0:9] = np.asarray(cam.R, np.float32).reshape(9)
    a[9:12] = np.asarray(cam.t, np.float32)
    a[12:17] = [cam.fx, cam.fy, cam.cx, cam.cy, cam.znear]
    return a.astype(dtype)


def _planes(planes, dtype):
    n = len(planes)
    arr = np.zeros((max(n, 1), 4), dtype)
    bits = np.zeros(max(n, 1), np.uint32)
    for k, (nrm, d, lb) in enumerate(planes):
        arr[k, :3] = np.asarray(nrm, np.float32)
        arr[k, 3] = np.float32(d)
        bits[k] = lb
    return np.ascontiguousarray(arr), bits, n


def sh_basis(deg: int, d, grad: bool = False):
    L = _load()
    d = _f64(d)
    Y = np.zeros(16)
    dY = np.zeros(48)
    L.or_sh_basis(deg, _p(d), _p(Y), _p(dY) if grad else None)
    K = (deg + 1) ** 2
    return (Y[:K], dY[:3 * K].reshape(K, 3)) if grad else Y[:K]


def quat_to_rot(q) -> np.ndarray:
    L = _load()
    q = _f64(q)
    R = np.zeros(9)
    L.or_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def expf32(x) -> np.ndarray:
    """The single-precision exponential of the decision path (elementwise)."""
    L = _load()
    x = np.asarray(x, np.float32).ravel()
    return np.array([L.or_expf32(float(v)) for v in x], np.float32)


def preprocess(scene, cam, layer_mask: int = 0xFFFFFFFF, planes=(), precision: str = "f64") -> dict:
    """Per-Gaussian projection: culls, screen mean, exponent coefficients, colour, rect.

    ``precision='f64'`` is the double-precision definition; ``'f32'`` is the
    single-precision decision path (fixed evaluation order).  Both return
    float64 arrays (the f32 values widened exactly)."""
    L = _load()
    n = scene.n
    W, H = int(cam.width), int(cam.height)
    out = dict(vis=np.zeros(n, np.int32), radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32))
    layer = np.ascontiguousarray(scene.layer, np.uint8)
    if precision == "f64":
        conv, dt = _f64, np.float64
    elif precision == "f32":
        conv, dt = _f32, np.float32
    else:
        raise ValueError(precision)
    for k in ("u", "v", "depth", "A2", "beta", "G2", "opac"):
        out[k] = np.zeros(n, dt)
    out["rgb"] = np.zeros((n, 3), dt)
    m, ls, q, ol, sh = (conv(scene.means), conv(scene.log_scales), conv(scene.quats),
                        conv(scene.opacity_logit), conv(scene.sh))
    pl, pb, npl = _planes(planes, dt)
    ca = cam_array(cam, dt)
    args = [n, _p(m), _p(ls), _p(q), _p(ol), _p(sh), _p(layer), int(scene.sh_degree), _p(ca), W, H,
            int(layer_mask) & 0xFFFFFFFF, _p(pl), _p(pb), npl,
            _p(out["vis"]), _p(out["u"]), _p(out["v"]), _p(out["depth"]), _p(out["A2"]), _p(out["beta"]),
            _p(out["G2"]), _p(out["opac"]), _p(out["rgb"]), _p(out["radius"]), _p(out["rect"])]
    if precision == "f64":
        out["cov2d"] = np.zeros((n, 3))
        L.or_preprocess64(*args, _p(out["cov2d"]))
    else:
        L.or_preprocess32(*args)
        for k in ("u", "v", "depth", "A2", "beta", "G2", "opac", "rgb"):
            out[k + "_f32"] = out[k]
            out[k] = out[k].astype(np.float64)
    out["tiles"] = np.where(out["vis"] > 0, (out["rect"][:, 2] - out["rect"][:, 0]) *
                            (out["rect"][:, 3] - out["rect"][:, 1]), 0).astype(np.int64)
    out["W"], out["H"] = W, H
    return out


def bin_tiles(pre: dict):
    """Tile lists ordered by (depth, index): returns ranges int64 [T,2] and list int32 [D]."""
    L = _load()
    W, H = pre["W"], pre["H"]
    n = pre["vis"].shape[0]
    Tn = ((W + TILE - 1) // TILE) * ((H + TILE - 1) // TILE)
    D = int(L.or_count_dups(n, _p(pre["vis"]), _p(pre["rect"])))
    ranges = np.zeros((Tn, 2), np.int64)
    lst = np.zeros(max(D, 1), np.int32)
    depth = _f64(pre["depth"])
    L.or_bin(n, _p(pre["vis"]), _p(pre["rect"]), _p(depth), W, H, _p(ranges), _p(lst))
    return ranges, lst[:D]


def composite(pre: dict, ranges, lst, bg=(0.0, 0.0, 0.0)) -> dict:
    L = _load()
    W, H = pre["W"], pre["H"]
    P = W * H
    o = dict(image=np.zeros((3, H, W)), alpha=np.zeros((H, W)), ncontrib=np.zeros((H, W), np.int64),
             T=np.zeros((H, W)), fragile=np.zeros((H, W), np.int32), alt_image=np.zeros((3, H, W)),
             alt_alpha=np.zeros((H, W)), alt_ncontrib=np.zeros((H, W), np.int64),
             dhash=np.zeros((H, W), np.uint64))
    lst = np.ascontiguousarray(lst, np.int32)
    if lst.size == 0:
        lst = np.zeros(1, np.int32)
    bgv = _f64(bg)
    L.or_composite(W, H, _p(np.ascontiguousarray(ranges, np.int64)), _p(lst), _p(_f64(pre["u"])),
                   _p(_f64(pre["v"])), _p(_f64(pre["A2"])), _p(_f64(pre["beta"])), _p(_f64(pre["G2"])),
                   _p(_f64(pre["opac"])), _p(_f64(pre["rgb"])), _p(bgv), _p(o["image"]), _p(o["alpha"]),
                   _p(o["ncontrib"]), _p(o["T"]), _p(o["fragile"]), _p(o["alt_image"]),
                   _p(o["alt_alpha"]), _p(o["alt_ncontrib"]), _p(o["dhash"]))
    del P
    return o


def composite_bruteforce(pre: dict, bg=(0.0, 0.0, 0.0)) -> dict:
    """Every visible Gaussian at every pixel in (depth, index) order (no tiles)."""
    L = _load()
    W, H = pre["W"], pre["H"]
    vis = np.nonzero(pre["vis"])[0]
    order = vis[np.lexsort((vis, pre["depth"][vis]))].astype(np.int32)
    order = np.ascontiguousarray(order) if order.size else np.zeros(1, np.int32)
    img, al = np.zeros((3, H, W)), np.zeros((H, W))
    L.or_composite_bruteforce(W, H, pre["vis"].shape[0], _p(order), int(vis.size), _p(_f64(pre["u"])),
                              _p(_f64(pre["v"])), _p(_f64(pre["A2"])), _p(_f64(pre["beta"])),
                              _p(_f64(pre["G2"])), _p(_f64(pre["opac"])), _p(_f64(pre["rgb"])),
                              _p(_f64(bg)), _p(img), _p(al))
    return dict(image=img, alpha=al)


def composite_pixels(pre: dict, ranges, lst, xs, ys, bg=(0.0, 0.0, 0.0)) -> dict:
    """or_composite at selected pixels only: rgb [k,3], alpha, ncontrib, fragile and alternatives."""
    L = _load()
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    k = xs.shape[0]
    if ys.shape != xs.shape or (k and (xs.min() < 0 or xs.max() >= pre["W"] or ys.min() < 0 or ys.max() >= pre["H"])):
        raise ValueError("composite_pixels: pixel coordinates outside the %dx%d frame" % (pre["W"], pre["H"]))
    o = dict(rgb=np.zeros((k, 3)), alpha=np.zeros(k), ncontrib=np.zeros(k, np.int64),
             fragile=np.zeros(k, np.int32), alt_rgb=np.zeros((k, 3)), alt_alpha=np.zeros(k),
             alt_ncontrib=np.zeros(k, np.int64))
    lst = np.ascontiguousarray(lst, np.int32)
    if lst.size == 0:
        lst = np.zeros(1, np.int32)
    L.or_composite_pixels(pre["W"], pre["H"], _p(np.ascontiguousarray(ranges, np.int64)), _p(lst),
                          _p(_f64(pre["u"])), _p(_f64(pre["v"])), _p(_f64(pre["A2"])), _p(_f64(pre["beta"])),
                          _p(_f64(pre["G2"])), _p(_f64(pre["opac"])), _p(_f64(pre["rgb"])), _p(_f64(bg)), k,
                          _p(xs), _p(ys), _p(o["rgb"]), _p(o["alpha"]), _p(o["ncontrib"]), _p(o["fragile"]),
                          _p(o["alt_rgb"]), _p(o["alt_alpha"]), _p(o["alt_ncontrib"]))
    return o


def composite_backward(pre: dict, ranges, lst, bg, dL_dimage, dL_dalpha=None, tile_mask=None) -> dict:
    """Record gradient [N,9] = d/d(u, v, A2, beta, G2, opac, r, g, b) and contributions
    (contrib_sum, contrib_max, and contrib_count: the number of pixels, i.e. of
    terms of contrib_sum, at which each Gaussian was blended).

    ``tile_mask`` (uint8 per tile) restricts the pass to the marked tiles."""
    L = _load()
    W, H = pre["W"], pre["H"]
    n = pre["vis"].shape[0]
    rg = np.zeros((n, 9))
    cs, cm = np.zeros(n), np.zeros(n)
    tf = np.zeros(n, np.int32)
    cc = np.zeros(n, np.int64)
    lst = np.ascontiguousarray(lst, np.int32)
    if lst.size == 0:
        lst = np.zeros(1, np.int32)
    dli = _f64(dL_dimage).reshape(3, H, W)
    dla = _f64(dL_dalpha).reshape(H, W) if dL_dalpha is not None else np.zeros((H, W))
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8).reshape(-1)
    if tm is not None and tm.size != np.asarray(ranges).shape[0]:
        raise ValueError("composite_backward: tile_mask needs one entry per tile (%d)" % np.asarray(ranges).shape[0])
    L.or_composite_backward(W, H, n, _p(np.ascontiguousarray(ranges, np.int64)), _p(lst),
                            _p(_f64(pre["u"])), _p(_f64(pre["v"])), _p(_f64(pre["A2"])),
                            _p(_f64(pre["beta"])), _p(_f64(pre["G2"])), _p(_f64(pre["opac"])),
                            _p(_f64(pre["rgb"])), _p(_f64(bg)), _p(dli), _p(dla), _p(tm) if tm is not None else None,
                            _p(rg), _p(cs), _p(cm), _p(tf), _p(cc))
    return dict(rec_grad=rg, contrib_sum=cs, contrib_max=cm, touched_fragile=tf, contrib_count=cc)


def chain(scene, cam, vis, rec_grad, grad_layer_mask: int = 0xFFFFFFFF) -> dict:
    """Chain rule from record gradients to (means, log_scales, quats, opacity_logit, sh)."""
    L = _load()
    n = scene.n
    K = (scene.sh_degree + 1) ** 2
    g = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), sh=np.zeros((n, K, 3)))
    L.or_chain(n, _p(_f64(scene.means)), _p(_f64(scene.log_scales)), _p(_f64(scene.quats)),
               _p(_f64(scene.opacity_logit)), _p(_f64(scene.sh)),
               _p(np.ascontiguousarray(scene.layer, np.uint8)), int(scene.sh_degree),
               _p(cam_array(cam)), int(cam.width), int(cam.height),
               _p(np.ascontiguousarray(vis, np.int32)), _p(_f64(rec_grad)),
               int(grad_layer_mask) & 0xFFFFFFFF, _p(g["means"]), _p(g["log_scales"]),
               _p(g["quats"]), _p(g["opacity_logit"]), _p(g["sh"]))
    return g


def prune(contrib_max, threshold: float = 0.005):
    L = _load()
    cm = _f64(contrib_max)
    keep = np.zeros(cm.shape[0], np.uint8)
    k = int(L.or_prune(cm.shape[0], _p(cm), float(threshold), _p(keep)))
    return keep, k


def render(scene, cam, layer_mask=0xFFFFFFFF, planes=(), bg=(0.0, 0.0, 0.0), precision="f64") -> dict:
    """Full forward: preprocess -> tile binning -> compositing."""
    pre = preprocess(scene, cam, layer_mask, planes, precision)
    ranges, lst = bin_tiles(pre)
    out = composite(pre, ranges, lst, bg)
    out.update(pre=pre, ranges=ranges, list=lst)
    return out


def render_backward(scene, cam, fwd: dict, bg, dL_dimage, dL_dalpha=None,
                    grad_layer_mask=0xFFFFFFFF, tile_mask=None) -> dict:
    """Analytic gradients of the render (FP64), plus per-Gaussian contributions."""
    pre = fwd["pre"]
    cb = composite_backward(pre, fwd["ranges"], fwd["list"], bg, dL_dimage, dL_dalpha, tile_mask)
    g = chain(scene, cam, pre["vis"], cb["rec_grad"], grad_layer_mask)
    g.update(cb)
    return g

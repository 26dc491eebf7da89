"""Saving and loading layered scenes and training state.

The paper trains one Gaussian cloud per anatomical layer and then
consolidates them into a single cloud whose points carry a layer property
next to their colour and scale attributes, stored as a PLY file (Sec. 3.2,
"Layered Training").  This module provides

* ``merge_layers``: that consolidation (clouds in layer order, each point
  tagged with its layer id);
* ``save_scene`` / ``load_scene``: a bit-exact archive (``.npz``) of a scene
  in its stored precision (FP32, FP16 or BF16 storage, or the SH codebook),
  host (``synth.Scene``) or device (``DeviceScene``);
* ``save_ply`` / ``load_ply``: the interchange format, binary little-endian
  PLY with the vertex properties of the 3DGS format the paper builds on
  (position, SH DC and higher-order coefficients channel by channel, opacity
  logit, log-scales, rotation quaternion) plus ``layer``; values are written
  as float32, so 16-bit storage is widened exactly;
* ``save_trainer`` / ``load_trainer``: everything a ``Trainer`` needs to
  resume: parameters, Adam moments and step, blend-weight and activity
  accumulators, the activity threshold and the configuration.

No arithmetic of the method happens here: arrays are copied byte for byte.
"""
from __future__ import annotations

import dataclasses
import json
from typing import Optional, Sequence

import numpy as np
import torch

FORMAT = 1
_SCENE_FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh", "layer")


# --------------------------------------------------------------------------- raw tensor bytes

def _to_bytes(t) -> tuple:
    """(uint8 bytes, dtype name, shape) of a torch tensor or numpy array."""
    if isinstance(t, np.ndarray):
        a = np.ascontiguousarray(t)
        return a.view(np.uint8).reshape(-1), "np:" + a.dtype.str, list(a.shape)
    t = t.detach().contiguous()
    return t.view(torch.uint8).reshape(-1).cpu().numpy(), "torch:" + str(t.dtype).replace("torch.", ""), \
        list(t.shape)


def _from_bytes(raw: np.ndarray, dtype: str, shape, device=None):
    kind, name = dtype.split(":", 1)
    if kind == "np":
        return np.frombuffer(raw.tobytes(), dtype=np.dtype(name)).reshape(shape).copy()
    t = torch.from_numpy(np.ascontiguousarray(raw)).view(getattr(torch, name)).reshape(shape)
    return t.to(device) if device is not None else t.clone()


def _pack(arrays: dict, meta: dict) -> dict:
    out = {}
    index = {}
    for k, v in arrays.items():
        raw, dt, shape = _to_bytes(v)
        out["a_" + k] = raw
        index[k] = [dt, shape]
    meta = dict(meta, format=FORMAT, arrays=index)
    out["meta"] = np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8)
    return out


def _unpack(path: str, device=None):
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError("%s: unknown checkpoint format %r" % (path, meta.get("format")))
        arrays = {k: _from_bytes(z["a_" + k], dt, shape, device) for k, (dt, shape) in meta["arrays"].items()}
    return arrays, meta


# --------------------------------------------------------------------------- scenes

def _is_device_scene(scene) -> bool:
    return hasattr(scene, "c_struct")


def merge_layers(parts: Sequence, layer_ids: Optional[Sequence[int]] = None):
    """One cloud from per-layer clouds (Sec. 3.2): the points of parts[k],
    all tagged with layer layer_ids[k] (default k), concatenated in order.
    Host scenes give a host scene, device scenes a device scene; all parts
    must share the SH degree and storage."""
    if not parts:
        raise ValueError("no layers to merge")
    ids = list(range(len(parts))) if layer_ids is None else [int(v) for v in layer_ids]
    if len(ids) != len(parts) or any(not 0 <= v < 32 for v in ids):
        raise ValueError("one layer id in 0..31 per part")
    deg = parts[0].sh_degree
    if any(p.sh_degree != deg for p in parts):
        raise ValueError("all layers must have the same SH degree")
    if _is_device_scene(parts[0]):
        from .api import DeviceScene
        if any(p.sh_dtype != parts[0].sh_dtype or p.sr_dtype != parts[0].sr_dtype for p in parts):
            raise ValueError("all layers must share their storage precision")
        if parts[0].sh_dtype == "cb":
            raise ValueError("codebook scenes are merged before encoding")
        cat = [torch.cat([getattr(p, f) for p in parts]).contiguous() for f in _SCENE_FIELDS[:5]]
        layer = torch.cat([torch.full((p.n,), v, dtype=torch.uint8, device=p.means.device)
                           for p, v in zip(parts, ids)])
        return DeviceScene(*cat, layer, deg, parts[0].sh_dtype, parts[0].sr_dtype)
    import synth
    cat = [np.concatenate([getattr(p, f) for p in parts]) for f in _SCENE_FIELDS[:5]]
    layer = np.concatenate([np.full(p.n, v, np.uint8) for p, v in zip(parts, ids)])
    return synth.Scene(*cat, layer, deg)


def save_scene(path: str, scene) -> None:
    """Writes ``scene`` (host or device) to ``path`` (.npz), every array in its
    stored dtype, byte for byte."""
    arrays = {f: getattr(scene, f) for f in _SCENE_FIELDS}
    meta = {"kind": "scene", "sh_degree": int(scene.sh_degree), "n": int(scene.n)}
    if _is_device_scene(scene):
        meta.update(sh_dtype=scene.sh_dtype, sr_dtype=scene.sr_dtype, device=True)
        if scene.sh_dtype == "cb":
            arrays.update(sh_index=scene.sh_index, sh_table=scene.sh_table)
    else:
        meta.update(sh_dtype="f32", sr_dtype="f32", device=False)
    np.savez(path, **_pack(arrays, meta))


def load_scene(path: str, device=None):
    """The scene saved at ``path``: a DeviceScene on ``device`` when given,
    else (for a host-saved scene) a synth.Scene.  The bytes of every array are
    those that were saved."""
    arrays, meta = _unpack(path, device)
    if meta.get("kind") != "scene":
        raise ValueError("%s holds no scene" % path)
    if device is None:
        if meta["device"]:
            raise ValueError("%s holds a device scene: pass device=" % path)
        import synth
        return synth.Scene(*(arrays[f] for f in _SCENE_FIELDS), meta["sh_degree"])
    from .api import DeviceScene
    if not meta["device"]:
        arrays = {k: torch.from_numpy(v).to(device) for k, v in arrays.items()}
    return DeviceScene(*(arrays[f] for f in _SCENE_FIELDS), meta["sh_degree"], meta["sh_dtype"], meta["sr_dtype"],
                       sh_index=arrays.get("sh_index"), sh_table=arrays.get("sh_table"))


# --------------------------------------------------------------------------- PLY

def _ply_props(K: int):
    names = ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"]
    names += ["f_rest_%d" % i for i in range(3 * (K - 1))]
    names += ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3"]
    return names


def _host_f32(scene):
    """(means, log_scales, quats, opacity_logit, sh, layer) as host float32 /
    uint8 arrays (16-bit storage widened exactly)."""
    if _is_device_scene(scene):
        if scene.sh_dtype == "cb":
            raise ValueError("PLY export of codebook scenes is not supported; save_scene keeps them")
        f = lambda t: t.detach().float().cpu().numpy()
        return (f(scene.means), f(scene.log_scales), f(scene.quats), f(scene.opacity_logit), f(scene.sh),
                scene.layer.cpu().numpy())
    return (np.asarray(scene.means, np.float32), np.asarray(scene.log_scales, np.float32),
            np.asarray(scene.quats, np.float32), np.asarray(scene.opacity_logit, np.float32),
            np.asarray(scene.sh, np.float32), np.asarray(scene.layer, np.uint8))


def save_ply(path: str, scene) -> None:
    """Binary little-endian PLY, one vertex per Gaussian: position, zero
    normal, SH (DC per channel, then the higher coefficients channel by
    channel), opacity logit, log-scales, quaternion (w, x, y, z) as float32,
    and the layer id as uchar."""
    means, ls, q, ol, sh, layer = _host_f32(scene)
    n = means.shape[0]
    K = sh.shape[1]
    names = _ply_props(K)
    cols = np.zeros((n, len(names)), np.float32)
    cols[:, 0:3] = means
    cols[:, 6:9] = sh[:, 0, :]
    if K > 1:
        cols[:, 9:9 + 3 * (K - 1)] = sh[:, 1:, :].transpose(0, 2, 1).reshape(n, -1)
    o = 9 + 3 * (K - 1)
    cols[:, o] = ol
    cols[:, o + 1:o + 4] = ls
    cols[:, o + 4:o + 8] = q
    rec = np.empty(n, dtype=[("f", "<f4", (len(names),)), ("layer", "u1")])
    rec["f"] = cols
    rec["layer"] = layer
    header = ["ply", "format binary_little_endian 1.0", "element vertex %d" % n]
    header += ["property float %s" % nm for nm in names]
    header += ["property uchar layer", "end_header"]
    with open(path, "wb") as fh:
        fh.write(("\n".join(header) + "\n").encode("ascii"))
        fh.write(rec.tobytes())


def load_ply(path: str):
    """A host synth.Scene from a PLY written by save_ply (or any binary
    little-endian 3DGS PLY; a missing layer property means layer 0)."""
    import synth
    with open(path, "rb") as fh:
        data = fh.read()
    end = data.index(b"end_header\n") + len(b"end_header\n")
    lines = data[:end].decode("ascii").splitlines()
    if lines[0] != "ply" or lines[1] != "format binary_little_endian 1.0":
        raise ValueError("%s: not a binary little-endian PLY" % path)
    n = None
    props = []
    for ln in lines[2:]:
        p = ln.split()
        if p[0] == "element":
            if p[1] != "vertex":
                break
            n = int(p[2])
        elif p[0] == "property":
            props.append((p[2], {"float": "<f4", "uchar": "u1", "double": "<f8"}[p[1]]))
    rec = np.frombuffer(data[end:end + n * np.dtype(props).itemsize], dtype=props, count=n)
    n_rest = sum(1 for nm, _ in props if nm.startswith("f_rest_"))
    K = 1 + n_rest // 3
    deg = int(round(K ** 0.5)) - 1
    if (deg + 1) ** 2 != K:
        raise ValueError("%s: %d SH coefficients per channel is not a full degree" % (path, K))
    g = lambda nm: np.ascontiguousarray(rec[nm], np.float32)
    means = np.stack([g("x"), g("y"), g("z")], 1)
    sh = np.zeros((n, K, 3), np.float32)
    for c in range(3):
        sh[:, 0, c] = g("f_dc_%d" % c)
        for k in range(1, K):
            sh[:, k, c] = g("f_rest_%d" % (c * (K - 1) + k - 1))
    ls = np.stack([g("scale_%d" % i) for i in range(3)], 1)
    q = np.stack([g("rot_%d" % i) for i in range(4)], 1)
    layer = np.ascontiguousarray(rec["layer"], np.uint8) if "layer" in rec.dtype.names else np.zeros(n, np.uint8)
    return synth.Scene(means, ls, q, g("opacity"), sh, layer, deg)


# --------------------------------------------------------------------------- training state

def save_trainer(path: str, trainer) -> None:
    """Everything a Trainer needs to resume: the scene, the Adam moments and
    step count, the blend-weight and activity accumulators, the activity
    threshold and sample count, and the configuration."""
    sc = trainer.scene
    arrays = {f: getattr(sc, f) for f in _SCENE_FIELDS}
    for k in range(5):
        arrays["m%d" % k] = trainer.m[k]
        arrays["v%d" % k] = trainer.v[k]
    arrays.update(contrib_max=trainer.contrib_max, contrib_sum=trainer.contrib_sum, activity=trainer.activity)
    meta = {"kind": "trainer", "sh_degree": int(sc.sh_degree), "n": int(sc.n), "t": int(trainer.t),
            "activity_samples": int(trainer.activity_samples),
            "activity_threshold": float(trainer.activity_threshold),
            "activity_removed": int(trainer.activity_removed), "dup_capacity": trainer.dup_capacity,
            "config": dataclasses.asdict(trainer.cfg)}
    np.savez(path, **_pack(arrays, meta))


def load_trainer(path: str, cameras, device="cuda"):
    """A Trainer restored from ``path`` on ``device`` with the given cameras;
    its next step continues the saved run."""
    from .api import DeviceScene
    from .train import TrainConfig, Trainer
    arrays, meta = _unpack(path, device)
    if meta.get("kind") != "trainer":
        raise ValueError("%s holds no training state" % path)
    cfg = meta["config"]
    cfg["lr"] = tuple(cfg["lr"])
    scene = DeviceScene(*(arrays[f] for f in _SCENE_FIELDS), meta["sh_degree"])
    tr = Trainer(scene, cameras, TrainConfig(**cfg), dup_capacity=meta["dup_capacity"])
    tr.m = [arrays["m%d" % k] for k in range(5)]
    tr.v = [arrays["v%d" % k] for k in range(5)]
    tr.t = meta["t"]
    tr.contrib_max, tr.contrib_sum, tr.activity = arrays["contrib_max"], arrays["contrib_sum"], arrays["activity"]
    tr.activity_samples = meta["activity_samples"]
    tr.activity_threshold = meta["activity_threshold"]
    tr.activity_removed = meta["activity_removed"]
    return tr

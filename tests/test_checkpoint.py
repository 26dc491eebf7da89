"""Saving and loading of layered scenes on the host: the .npz archive keeps
every array byte for byte; the consolidation of per-layer clouds into one
cloud with a layer property (Sec. 3.2) keeps each layer's points in order;
the PLY interchange file round-trips exactly and carries the layer ids."""
import numpy as np
import pytest

import synth
from paper_2410_16978_gb300 import checkpoint as ck

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh", "layer")


def _same(a, b):
    for f in FIELDS:
        x, y = getattr(a, f), getattr(b, f)
        assert x.dtype == y.dtype and x.shape == y.shape, f
        assert np.array_equal(np.ascontiguousarray(x).view(np.uint8), np.ascontiguousarray(y).view(np.uint8)), f
    assert a.sh_degree == b.sh_degree


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_scene_archive_round_trip_is_bit_exact(which, tmp_path):
    sc = synth.scene_c1()["scene"] if which == "c1" else synth.scene_c2(scale=0.01)["scene"]
    sc.means[0, 0] = np.float32(-0.0)                  # signed zero and a subnormal survive
    sc.opacity_logit[1] = np.float32(1e-40)
    p = str(tmp_path / "scene.npz")
    ck.save_scene(p, sc)
    _same(sc, ck.load_scene(p))


def test_merge_layers_tags_each_cloud_with_its_layer():
    w = synth.scene_c2(scale=0.01)
    sc = w["scene"]
    parts = [sc.subset(np.nonzero(sc.layer == L)[0]) for L in range(5)]
    merged = ck.merge_layers(parts)
    _same(sc, merged)                                   # the workload's layers are contiguous, in order
    m2 = ck.merge_layers(parts[:2], layer_ids=[7, 3])
    assert np.array_equal(m2.layer, np.r_[np.full(parts[0].n, 7), np.full(parts[1].n, 3)].astype(np.uint8))
    with pytest.raises(ValueError):
        ck.merge_layers([synth.scene_c1()["scene"], sc])          # SH degree 0 and 3
    with pytest.raises(ValueError):
        ck.merge_layers(parts[:2], layer_ids=[0, 32])


@pytest.mark.parametrize("deg", [0, 3])
def test_ply_round_trip_and_layout(deg, tmp_path):
    sc = synth.scene_c1()["scene"] if deg == 0 else synth.scene_c2(scale=0.005)["scene"]
    sc = ck.merge_layers([sc.subset(np.arange(0, sc.n // 2)), sc.subset(np.arange(sc.n // 2, sc.n))], [4, 9])
    p = str(tmp_path / "scene.ply")
    ck.save_ply(p, sc)
    _same(sc, ck.load_ply(p))
    head = open(p, "rb").read(4096).split(b"end_header\n")[0].decode().splitlines()
    K = (deg + 1) ** 2
    props = [ln.split()[-1] for ln in head if ln.startswith("property")]
    assert head[2] == "element vertex %d" % sc.n
    assert props[:9] == ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"]
    assert props[9:9 + 3 * (K - 1)] == ["f_rest_%d" % i for i in range(3 * (K - 1))]
    assert props[-9:] == ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3", "layer"]
    # the higher SH coefficients are written channel by channel: f_rest_0 is coefficient 1 of red
    if deg:
        raw = open(p, "rb").read()
        body = raw[raw.index(b"end_header\n") + 11:]
        rec = np.frombuffer(body, dtype=[("f", "<f4", (len(props) - 1,)), ("l", "u1")], count=sc.n)
        assert rec["f"][0, 9] == sc.sh[0, 1, 0] and rec["f"][0, 9 + K - 1] == sc.sh[0, 1, 1]


def test_ply_without_layer_property_loads_as_layer_zero(tmp_path):
    sc = synth.scene_c1(scale=0.01)["scene"]
    p = str(tmp_path / "a.ply")
    ck.save_ply(p, sc)
    raw = open(p, "rb").read()
    end = raw.index(b"end_header\n") + 11
    head = raw[:end].replace(b"property uchar layer\n", b"")
    n = sc.n
    row = (len(raw) - end) // n
    body = b"".join(raw[end + i * row:end + (i + 1) * row - 1] for i in range(n))
    q = str(tmp_path / "b.ply")
    open(q, "wb").write(head + body)
    back = ck.load_ply(q)
    assert np.array_equal(back.layer, np.zeros(n, np.uint8))
    assert np.array_equal(back.means, sc.means)

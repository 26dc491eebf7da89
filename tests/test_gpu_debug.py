"""The GS_DEBUG build (libgs_debug.so) on the GPU: its bounds checks stay
silent on valid scenes and give the release build's images; a check that
fails reports GS_ERR_BOUNDS and the check's site through the status word and
skips the access; and the depth sort's bounded look-back wait, made to run
out by its test hook, ends in GS_ERR_TIMEOUT with the context still usable.

No test here faults or hangs the GPU: the only out-of-range value (a
corrupted list entry) is read by the debug build alone, whose check skips
it, and every wait has an iteration limit."""
import numpy as np
import pytest
import torch

import synth
from paper_2410_16978_gb300 import DeviceScene, Rasterizer, _lib
from tests.helpers import branch_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    lib = _lib.load_debug()
    assert lib.gs_debug_build() == 1
    return lib


def _render(ds, cam, mask, planes, bg, check=True):
    r = Rasterizer(ds.n, cam.width, cam.height)
    img, al = r.render(ds, cam, mask, planes, bg, check=check)
    torch.cuda.synchronize()
    return r, img, al


def _scenes():
    w = synth.scene_c2(scale=0.05, width=512, height=512)
    sc, cam, planes, _ = branch_scene()
    return [(w["scene"], w["cameras"][0], w["layer_mask"], w["planes"]), (sc, cam, 0xFFFFFFFF, planes)]


def test_debug_build_is_silent_and_matches_release(dbg):
    for sc, cam, mask, planes in _scenes():
        ds = DeviceScene.from_host(sc)
        bg = (0.1, 0.2, 0.3)
        _, img_r, al_r = _render(ds, cam, mask, planes, bg)
        rng = np.random.default_rng(1)
        dimg = torch.from_numpy(rng.standard_normal((3, cam.height, cam.width)).astype(np.float32)).cuda()
        with _lib.use(dbg):
            r, img_d, al_d = _render(ds, cam, mask, planes, bg)
            g = r.backward(ds, cam, bg, dimg)
            st = r.status()
            site = _lib.gs_debug_site(r.workspace, 0)
        assert st.error == _lib.GS_OK and site == 0
        assert torch.equal(img_r, img_d) and torch.equal(al_r, al_d)
        assert all(bool(torch.isfinite(v).all()) for v in g.values())


def test_failed_bounds_check_reports_and_skips(dbg):
    """A pair-list entry overwritten with an id far beyond the scene: the
    debug backward's check rejects it (GS_ERR_BOUNDS, site 8: a Gaussian id
    read by the backward compositor) and treats the entry as transparent."""
    w = synth.scene_c2(scale=0.02, width=256, height=256)
    sc, cam = w["scene"], w["cameras"][0]
    ds = DeviceScene.from_host(sc)
    bg = (0.0, 0.0, 0.0)
    with _lib.use(dbg):
        r, img, al = _render(ds, cam, w["layer_mask"], w["planes"], bg)
        lay = _lib.gs_workspace_layout(r.n, cam.width, cam.height, r.ws_bytes)
        Tn = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
        ranges = r.workspace[lay["ranges"]:lay["ranges"] + 8 * Tn].view(torch.int32).view(Tn, 2).cpu().numpy()
        ncon = r.workspace[lay["n_contrib"]:lay["n_contrib"] + 4 * cam.width * cam.height].view(torch.int32)
        ncon = ncon.view(cam.height, cam.width).cpu().numpy()
        Tx = (cam.width + 15) // 16
        # a tile with blended splats: every entry of its blended prefix is overwritten, so the backward
        # reads at least one bad id (an entry that some pixel blended)
        tile = next(t for t in range(Tn) if ranges[t, 1] > ranges[t, 0] and
                    ncon[(t // Tx) * 16:(t // Tx) * 16 + 16, (t % Tx) * 16:(t % Tx) * 16 + 16].max() >= 1)
        pos = int(ranges[tile, 0])
        k = int(ncon[(tile // Tx) * 16:(tile // Tx) * 16 + 16, (tile % Tx) * 16:(tile % Tx) * 16 + 16].max())
        bad = torch.full((k,), 0xFFFFFFF0, dtype=torch.int64).to(torch.int32).view(torch.uint8).cuda()
        r.workspace[lay["list"] + 4 * pos:lay["list"] + 4 * (pos + k)].copy_(bad)
        g = r.backward(ds, cam, bg, torch.ones((3, cam.height, cam.width), device="cuda"))
        torch.cuda.synchronize()
        st = r.status()
        site = _lib.gs_debug_site(r.workspace, 0)
    assert st.error == _lib.GS_ERR_BOUNDS
    assert site == 8
    assert all(bool(torch.isfinite(v).all()) for v in g.values())


def test_sort_wait_runs_out_with_timeout_status(dbg):
    """The first tile of the second digit kernel never publishes its counts:
    every later tile waits for it until the (shortened) limit runs out.  The
    status word then holds GS_ERR_TIMEOUT, the binning leaves the unfinished
    order alone (nothing is drawn), and after the hook is reset the same
    workspace renders the release build's image again."""
    w = synth.scene_c2(scale=0.1, width=512, height=512)
    sc, cam = w["scene"], w["cameras"][0]
    ds = DeviceScene.from_host(sc)
    bg = (0.25, 0.5, 0.75)
    _, img_ref, al_ref = _render(ds, cam, w["layer_mask"], w["planes"], bg)
    with _lib.use(dbg):
        r, _, _ = _render(ds, cam, w["layer_mask"], w["planes"], bg)     # sizes the pair list
        assert r.status().n_visible > 3 * 4096     # several tiles in the digit kernels after the first
        try:
            _lib.gs_debug_sort_wait(2000, 1)
            img, al = r.render(ds, cam, w["layer_mask"], w["planes"], bg, check=False)
            torch.cuda.synchronize()
            st = r.status()
            assert st.error == _lib.GS_ERR_TIMEOUT
            assert float(al.abs().max()) == 0.0
            for c in range(3):
                assert bool((img[c] == bg[c]).all())
            with pytest.raises(_lib.GsError) as e:
                r.render(ds, cam, w["layer_mask"], w["planes"], bg, check=True)
            assert e.value.code == _lib.GS_ERR_TIMEOUT
        finally:
            _lib.gs_debug_sort_wait(0, -1)
        img2, al2 = r.render(ds, cam, w["layer_mask"], w["planes"], bg, check=True)
        torch.cuda.synchronize()
        assert r.status().error == _lib.GS_OK
    assert torch.equal(img2, img_ref) and torch.equal(al2, al_ref)

"""The contribution prune without a caller workspace (gs_contrib_prune_noalloc).

Some users of this library cannot allocate device memory when they prune: a
plugin that runs inside a host application's per-frame render callback (a
game engine or VR compositor), where cudaMalloc would synchronise the device
and stall the frame or is not permitted at all, or a service that reserves
all of its device memory once at start-up.  This entry point keeps its scan
scratch in a static array inside the library instead.  The test calls it
through the C ABI twice in a row (the second call reuses the scratch the first
one left behind, with a smaller input) and requires the same keep mask, kept
indices and count as gs_contrib_prune with its own workspace."""
import numpy as np
import pytest
import torch

from paper_2410_16978_gb300 import _lib

pytestmark = pytest.mark.gpu


def _stream():
    return int(torch.cuda.current_stream().cuda_stream)


def _outputs(n):
    return (torch.empty(n, dtype=torch.uint8, device="cuda"), torch.full((n,), -1, dtype=torch.int32, device="cuda"),
            torch.full((1,), -1, dtype=torch.int64, device="cuda"))


def _with_workspace(cm, thr):
    n = cm.numel()
    keep, idx, nk = _outputs(n)
    wsb = _lib.gs_prune_workspace_size(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    _lib.gs_contrib_prune(cm, n, thr, keep, idx, nk, ws, wsb, _stream())
    return keep, idx, nk


def _without_workspace(cm, thr):
    n = cm.numel()
    keep, idx, nk = _outputs(n)
    _lib.gs_contrib_prune_noalloc(cm, n, thr, keep, idx, nk, _stream())
    return keep, idx, nk


def test_noalloc_prune_warm_up_call_with_no_items():
    # The set-up call a caller that may not allocate later makes once per
    # device: it loads the module (backing the static array) and writes a
    # count of zero.
    keep, idx, nk = _outputs(1)
    _lib.gs_contrib_prune_noalloc(keep, 0, 0.005, keep, idx, nk, _stream())
    torch.cuda.synchronize()
    assert int(nk.item()) == 0


def test_noalloc_prune_matches_workspace_prune_on_two_calls_in_a_row():
    rng = np.random.default_rng(20241022)
    for n, thr in ((300_001, 0.005), (70_000, 0.002)):
        cm_h = rng.uniform(0.0, 0.01, n).astype(np.float32)
        cm_h[:7] = np.float32(thr)                                  # exactly at the threshold: kept
        cm = torch.from_numpy(cm_h).cuda()
        k_ref, i_ref, n_ref = _with_workspace(cm, thr)
        k_new, i_new, n_new = _without_workspace(cm, thr)
        torch.cuda.synchronize()
        count = int(n_ref.item())
        assert int(n_new.item()) == count
        assert 0 < count < n
        assert torch.equal(k_new, k_ref)
        assert torch.equal(i_new[:count], i_ref[:count])


def test_noalloc_prune_rejects_counts_beyond_its_scratch():
    keep, idx, nk = _outputs(1)
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_contrib_prune_noalloc(keep, 1 << 31, 0.005, keep, idx, nk, _stream())
    assert e.value.code == _lib.GS_ERR_INVALID
    assert "static" in _lib.gs_last_error_string()

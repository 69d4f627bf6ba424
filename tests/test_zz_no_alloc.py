"""gs_bin_sort_noalloc: the binning sort for callers that cannot allocate.

Some callers of this library cannot allocate device memory (a runtime that
owns every device allocation through its own pool, a steady-state loop that
must not call cudaMalloc/cudaFree because they can synchronise the device).
gs_bin_sort_noalloc serves them: it takes no workspace and keeps its scratch
in a fixed device array inside the library.  This file checks, through the C
ABI, that two calls in a row give exactly what gs_bin_sort gives with a
caller-allocated workspace (the outputs are integers: bit for bit), and that a
problem larger than the fixed scratch is refused.  It is collected last, and
passes on its own in a fresh process as well.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _project(scene, cam):
    params = P.to_device_params(scene)
    views = P.param_views(params, scene.n)
    fr = P.Frame([cam], scene.n)
    fr.project(views)
    return fr


def _with_workspace(fr, cam, n, cap):
    vals = torch.zeros(cap, dtype=torch.int32, device="cuda")
    ranges = torch.zeros(2 * cam.n_tiles, dtype=torch.int32, device="cuda")
    ninst = torch.zeros(1, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(L.gs_bin_sort_workspace([cam], n, cap) // 4 + 64, dtype=torch.float32, device="cuda")
    L.gs_bin_sort([cam], n, fr.depth, fr.rect, fr.touched, cap, vals, ranges, None, ninst, ws, err)
    return vals, ranges, ninst, err


def _noalloc_c_abi(fr, cam, n, cap):
    """Call the entry point directly through ctypes (plain pointers)."""
    vals = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    ranges = torch.full((2 * cam.n_tiles,), -7, dtype=torch.int32, device="cuda")
    ninst = torch.zeros(1, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    cams = L.camera_array([cam])
    rc = L.lib().gs_bin_sort_noalloc(cams, 1, n, fr.depth.data_ptr(), fr.rect.data_ptr(),
                                     fr.touched.data_ptr(), ctypes.c_longlong(cap), vals.data_ptr(),
                                     ranges.data_ptr(), None, ninst.data_ptr(), err.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream or None)
    return rc, vals, ranges, ninst, err


def test_noalloc_matches_workspace_version_twice():
    cam = S.front_camera(256, 256)
    for seed in (0, 1):                       # two calls in a row share the fixed scratch
        scene = S.uniform_scene(10_000, seed)
        fr = _project(scene, cam)
        ref_vals, ref_ranges, ref_n, ref_err = _with_workspace(fr, cam, scene.n, 60_000)
        rc, vals, ranges, ninst, err = _noalloc_c_abi(fr, cam, scene.n, 60_000)
        torch.cuda.synchronize()
        assert rc == L.GS_OK
        n = int(ref_n.item())
        assert n > 0 and int(ninst.item()) == n
        assert int(err.item()) == int(ref_err.item()) == 0
        assert torch.equal(ranges, ref_ranges)
        assert torch.equal(vals[:n], ref_vals[:n])


def test_noalloc_refuses_problems_beyond_its_scratch():
    cam = S.front_camera(1600, 1060)
    n, cap = 3_000_000, 150_000_000
    need = L.gs_bin_sort_workspace([cam], n, cap)
    assert need > (32 << 20)
    cams = L.camera_array([cam])
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    p = dummy.data_ptr()
    rc = L.lib().gs_bin_sort_noalloc(cams, 1, n, p, p, p, ctypes.c_longlong(cap), p, p, None, p, p, None)
    assert rc == L.GS_ERR_CAPACITY

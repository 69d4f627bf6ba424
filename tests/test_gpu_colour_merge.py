"""Similarity-based sampling and merging of tile lists (Sec. IV-C1) on the
GPU against the oracle (needs a GPU).

gs_colour_merge groups each tile's entries by colour bucket and keeps one
representative per bucket (the first in depth order, with the bucket's mean
colour and accumulated opacity); gs_render_fwd then renders the merged
lists.  The oracle (O.colour_merge, O.render_lists) does the same from the
FP64 projection.  Which entries represent which buckets, and how many members
each stands for, must match exactly: the record colours are the same on both
sides (16-bit records of a storage-prepared scene, or FP32 records of a
scene whose colours keep clear of the hash's quantisation steps).  The merged
image matches the oracle's merged image within 1e-4 on unflagged pixels.  Its
distance to the exact image (the method is lossy) is printed, not bounded."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import IMG_ATOL, oracle_lists, storage_refs, storage_scene

pytestmark = pytest.mark.gpu

TDT = {L.GS_BF16: torch.bfloat16, L.GS_F16: torch.float16}
CASES = {
    "uniform-10k-256x256": lambda: (S.uniform_scene(10_000, 0), S.front_camera(256, 256)),
    "skewed-20k-200x136": lambda: (S.skewed_scene(20_000, 0), S.front_camera(200, 136)),
}


def _merged(fr, dtype):
    cap = fr.vals.numel()
    out = dict(ranges=torch.zeros(fr.T * 2, dtype=torch.int32, device="cuda"),
               vals=torch.zeros(cap, dtype=torch.int32, device="cuda"),
               splats=torch.zeros(cap * 12, dtype=torch.float32, device="cuda"),
               src=torch.zeros(cap, dtype=torch.int32, device="cuda"),
               members=torch.zeros(cap, dtype=torch.int32, device="cuda"))
    L.gs_colour_merge(fr.T, fr.ranges, fr.vals, fr.splats, dtype, out["ranges"], out["vals"], out["splats"],
                      out["src"], out["members"])
    img = torch.empty_like(fr.img)
    T_final = torch.empty_like(fr.T_final)
    n_proc = torch.empty_like(fr.n_proc)
    L.gs_render_fwd(fr.cams, out["ranges"], out["vals"], out["splats"], L.GS_F32, None, img, T_final, n_proc,
                    torch.empty_like(fr.tile_nproc), None, fr.err)
    torch.cuda.synchronize()
    return out, img


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", [L.GS_F32, L.GS_BF16, L.GS_F16], ids=["f32", "bf16", "f16"])
def test_merged_lists_and_image_match_oracle(case, dtype):
    scene, cam = CASES[case]()
    sc = storage_scene(scene, [cam], dtype, hash_safe=dtype == L.GS_F32)
    params = P.to_device_params(sc)
    views = dict(P.param_views(params, sc.n))
    if dtype != L.GS_F32:
        views["sh"] = views["sh"].to(TDT[dtype])
    fr = P.Frame([cam], sc.n, rgb_dtype=dtype, sh_dtype=dtype)
    fr.project(views)
    fr.bin_sort()
    out, img = _merged(fr, dtype)
    assert fr.check_errors() == 0
    # the oracle: lists, record colours, merge, render
    ref = storage_refs(sc, [cam], dtype)[0]
    kp, pr = ref["kp"], ref["proj"]
    vals_o, ranges_o = oracle_lists(cam, kp)
    rec_rgb = pr["rgb"].astype(np.float32)             # what a record holds (16-bit values are exact)
    mr, ids, reps, src, members = O.colour_merge(ranges_o, vals_o, rec_rgb, pr)
    # representatives: per tile the same Gaussians, in the same order, with the same member counts
    rg = out["ranges"].cpu().numpy().reshape(-1, 2).astype(np.int64)
    n_rep = rg[:, 1] - rg[:, 0]
    assert np.array_equal(n_rep, mr[:, 1] - mr[:, 0])
    g_src = out["src"].cpu().numpy()
    g_mem = out["members"].cpu().numpy()
    got_src = np.concatenate([g_src[a:b] for a, b in rg]) if n_rep.sum() else np.zeros(0)
    got_mem = np.concatenate([g_mem[a:b] for a, b in rg]) if n_rep.sum() else np.zeros(0)
    assert np.array_equal(got_src, src) and np.array_equal(got_mem, members)
    assert np.array_equal(out["vals"].cpu().numpy()[rg[n_rep > 0, 0]], rg[n_rep > 0, 0])
    # the merged image
    r = O.render_lists(cam, mr, ids, reps)
    ok = r["flag"] == 0
    assert ok.mean() > 0.98
    got = img.view(3, cam.H, cam.W).cpu().numpy()
    assert np.abs(got - r["img"])[:, ok].max() <= IMG_ATOL
    # how far the lossy merge moves the image from the exact one
    ex = ref["r"]["img"]
    err = np.abs(got - ex)
    mse = float(np.mean((got - ex) ** 2))
    print(f"\n{case} {dtype}: {len(src)} of {len(vals_o)} entries kept ({len(src) / max(1, len(vals_o)):.1%}); "
          f"merged vs exact image: max {err.max():.3e}, mean {err.mean():.3e}, "
          f"PSNR {10 * math.log10(1.0 / max(mse, 1e-30)):.1f} dB")


def test_merge_of_empty_lists():
    cam = S.front_camera(64, 48)
    T = cam.n_tiles
    ranges = torch.zeros(T * 2, dtype=torch.int32, device="cuda")
    vals = torch.zeros(4, dtype=torch.int32, device="cuda")
    splats = torch.zeros(4 * 12, dtype=torch.float32, device="cuda")
    out_r = torch.full((T * 2,), 7, dtype=torch.int32, device="cuda")
    out_v = torch.zeros(4, dtype=torch.int32, device="cuda")
    out_s = torch.zeros(4 * 12, dtype=torch.float32, device="cuda")
    L.gs_colour_merge(T, ranges, vals, splats, L.GS_F32, out_r, out_v, out_s)
    torch.cuda.synchronize()
    assert int(out_r.abs().sum()) == 0

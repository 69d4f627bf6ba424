"""Multi-view batches, storage precisions and edge cases on the GPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import GRAD_RTOL, IMG_ATOL, oracle_lists, rel_check

pytestmark = pytest.mark.gpu


def _frame(scene, cams, rgb=L.GS_F32, sh=L.GS_F32, schedule=None, keys=False):
    params = P.to_device_params(scene)
    views = dict(P.param_views(params, scene.n))
    if sh != L.GS_F32:
        views["sh"] = views["sh"].to(torch.bfloat16 if sh == L.GS_BF16 else torch.float16)
    fr = P.Frame(cams, scene.n, rgb_dtype=rgb, sh_dtype=sh, schedule=schedule)
    fr.project(views)
    fr.bin_sort(want_keys=keys)
    fr.render()
    torch.cuda.synchronize()
    return fr, views


def test_multi_view_batch_matches_per_view_oracle():
    scene = S.skewed_scene(12_000, 1)
    sizes = [(160, 120), (250, 170), (96, 200)]
    cams = S.ring_cameras(3, sizes)
    fr, views = _frame(scene, cams, keys=True)
    n = scene.n
    vals = fr.vals.cpu().numpy().view(np.uint32)
    ranges = fr.ranges.cpu().numpy().reshape(-1, 2).astype(np.int64)
    base = 0
    dimg = []
    refs = []
    for v, cam in enumerate(cams):
        kp = O.keypath(cam, scene)
        assert np.array_equal(fr.touched.cpu().numpy()[v * n:(v + 1) * n], kp["touched"])
        vo, ro = oracle_lists(cam, kp)
        for t in range(cam.n_tiles):
            a, b = ranges[base + t]
            assert np.array_equal(vals[a:b] - v * n, vo[ro[t, 0]:ro[t, 1]]), (v, t)
        base += cam.n_tiles
        pr = O.project(cam, scene, kp)
        r = O.render(cam, kp, pr)
        ok = r["flag"] == 0
        img = fr.image(v).cpu().numpy()
        assert np.abs(img - r["img"])[:, ok].max() <= IMG_ATOL
        d = S.random_cotangent((3, cam.H, cam.W), seed=10 + v) * 1e-3
        d[:, ~ok] = 0.0
        dimg.append(d.ravel())
        refs.append((kp, pr, d))
    # gradients summed over the views
    g = fr.backward(views, torch.from_numpy(np.concatenate(dimg)).cuda()).cpu().numpy()
    gref = np.zeros(59 * n)
    for cam, (kp, pr, d) in zip(cams, refs):
        gref += O.project_bwd(cam, scene, kp, O.render_bwd(cam, kp, pr, d.astype(np.float64)))
    rel_check(g[:3 * n].reshape(n, 3), gref[:3 * n].reshape(n, 3), GRAD_RTOL, "means")
    rel_check(g[11 * n:].reshape(n, 48), gref[11 * n:].reshape(n, 48), GRAD_RTOL, "sh")


@pytest.mark.parametrize("dtype", [L.GS_BF16, L.GS_F16])
def test_half_storage_parity(dtype):
    """SH and colours stored in 16 bits; blending and gradients in FP32.
    Parity: the oracle reads the same rounded SH; the colour rounding of the
    record adds at most half an ulp of the colour, so per pixel
    |img - oracle| <= 2^-p * oracle(|c|) + 1e-4 (p = 8 for BF16, 11 for FP16)."""
    scene = S.uniform_scene(10_000, 0)
    cam = S.front_camera(256, 256)
    fr, views = _frame(scene, [cam], rgb=dtype, sh=dtype)
    tdt = torch.bfloat16 if dtype == L.GS_BF16 else torch.float16
    sc16 = scene.subset(np.arange(scene.n))
    sc16.sh = torch.from_numpy(scene.sh).to(tdt).float().numpy()
    r = O.forward(cam, sc16)
    ok = r["flag"] == 0
    p = 8 if dtype == L.GS_BF16 else 11
    img = fr.image(0).cpu().numpy()
    bound = 2.0 ** -p * r["img"] + IMG_ATOL
    assert np.all(np.abs(img - r["img"])[:, ok] <= bound[:, ok])
    # accuracy against the FP32-SH oracle, reported
    r32 = O.forward(cam, scene)
    ok32 = ok & (r32["flag"] == 0)
    err = np.abs(img - r32["img"])[:, ok32]
    print(f"\n{'bf16' if dtype == L.GS_BF16 else 'fp16'} storage vs FP64 oracle on FP32 SH: "
          f"max {err.max():.3e}, mean {err.mean():.3e}")


def test_empty_and_all_culled():
    cam = S.front_camera(64, 48)
    fr = P.Frame([cam], 0)
    z = torch.zeros(4, device="cuda")
    fr.project({"means": z, "log_scales": z, "quats": z, "opacity_logits": z, "sh": z})
    fr.bin_sort()
    fr.render()
    torch.cuda.synchronize()
    assert int(fr.n_inst.item()) == 0
    assert torch.all(fr.image(0) == 0.0) and torch.all(fr.T_final == 1.0)
    scene = S.uniform_scene(400, 2)
    scene.means[:, 2] = -3.5                                  # all behind the camera
    cam.bg = (0.1, 0.2, 0.3)
    fr, _ = _frame(scene, [cam])
    assert int(fr.n_inst.item()) == 0
    img = fr.image(0).cpu().numpy()
    for ch in range(3):
        assert np.all(img[ch] == np.float32(cam.bg[ch]))


def test_capacity_overflow_flag():
    scene = S.uniform_scene(3000, 4)
    cam = S.front_camera(128, 128)
    fr, views = _frame(scene, [cam])
    need = int(fr.n_inst.item())
    cap = need // 2
    vals = torch.full((need,), -1, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    nws = L.gs_bin_sort_workspace([cam], scene.n, cap)
    ws = torch.empty(nws // 4 + 64, dtype=torch.float32, device="cuda")
    ninst = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.gs_bin_sort([cam], scene.n, fr.depth, fr.rect, fr.touched, cap, vals, fr.ranges, None, ninst, ws, err)
    torch.cuda.synchronize()
    assert int(ninst.item()) == need
    assert int(err.item()) & L.GS_EW_CAPACITY
    assert torch.all(vals[cap:] == -1)                         # nothing written past the capacity


def test_nonfinite_parameter_is_culled_and_flagged():
    scene = S.uniform_scene(2000, 6)
    scene.means[7, 1] = np.nan
    scene.log_scales[11, 0] = np.inf
    cam = S.front_camera(96, 96)
    fr, _ = _frame(scene, [cam])
    assert fr.check_errors() & L.GS_EW_NONFINITE
    kp = O.keypath(cam, scene)
    assert kp["status"][7] == 1 and kp["status"][11] == 1
    t = fr.touched.cpu().numpy()
    assert t[7] == 0 and t[11] == 0 and np.array_equal(t, kp["touched"])
    r = O.render(cam, kp, O.project(cam, scene, kp))
    ok = r["flag"] == 0
    assert np.abs(fr.image(0).cpu().numpy() - r["img"])[:, ok].max() <= IMG_ATOL


def test_depth_ties_order_by_index():
    scene = S.uniform_scene(64, 3)
    scene.means[:, 2] = 0.0                                   # identical depths
    scene.log_scales[:] = -2.0
    cam = S.front_camera(64, 64)
    fr, _ = _frame(scene, [cam])
    kp = O.keypath(cam, scene)
    vo, ro = oracle_lists(cam, kp)
    I = int(fr.n_inst.item())
    assert np.array_equal(fr.vals.cpu().numpy()[:I].view(np.uint32), vo)


def test_whole_image_gaussian():
    scene = S.uniform_scene(8, 1)
    scene.means[:] = 0.0
    scene.log_scales[:] = 0.5                                 # covers every tile
    cam = S.front_camera(200, 120)
    fr, _ = _frame(scene, [cam])
    assert np.all(fr.touched.cpu().numpy() == cam.n_tiles)
    r = O.forward(cam, scene)
    ok = r["flag"] == 0
    assert np.abs(fr.image(0).cpu().numpy() - r["img"])[:, ok].max() <= IMG_ATOL


def test_timeout_budget_sets_error_without_hanging():
    scene = S.uniform_scene(20_000, 0)
    cam = S.front_camera(512, 512)
    fr, _ = _frame(scene, [cam])
    L.gs_range_cost(fr.ranges, fr.T, fr.cost)
    L.gs_sched_order(fr.cost, fr.T, fr.order_f, fr.order_ws)
    fr.err.zero_()
    sched = {"mode": L.GS_SCHED_ORDER, "order": fr.order_f, "queue": fr.queue, "budget_ns": 1}
    L.gs_render_fwd(fr.cams, fr.ranges, fr.vals, fr.splats, fr.rgb_dtype, sched, fr.img, fr.T_final,
                    fr.n_proc, fr.tile_nproc, None, fr.err)
    torch.cuda.synchronize()
    assert fr.check_errors() & L.GS_EW_TIMEOUT


def test_depth_sort_wait_limit_sets_error_and_returns():
    """The onesweep depth sort's look-back reads are bounded (gs_set_wait_limit).
    At 0 every tile after the first gives up at once: the call returns,
    GS_EW_TIMEOUT is set, and the lists it leaves hold record indices only.
    With the default limit restored the same call is exact again."""
    scene = S.uniform_scene(10_000, 0)           # 10k records: three 4096-key tiles per digit pass
    cam = S.front_camera(256, 256)
    fr, _ = _frame(scene, [cam])
    I = int(fr.n_inst.item())
    want = fr.vals[:I].clone()
    assert L.gs_get_wait_limit() == 1 << 20 and fr.check_errors() == 0
    try:
        L.gs_set_wait_limit(0)
        assert L.gs_get_wait_limit() == 0
        fr.err.zero_()
        fr.bin_sort()
        torch.cuda.synchronize()
        assert fr.check_errors() & L.GS_EW_TIMEOUT
        got = fr.vals[:min(I, fr.capacity)]
        assert int(got.min()) >= 0 and int(got.max()) < scene.n
    finally:
        L.gs_set_wait_limit(1 << 20)
    fr.err.zero_()
    fr.bin_sort()
    torch.cuda.synchronize()
    assert fr.check_errors() == 0
    assert int(fr.n_inst.item()) == I and torch.equal(fr.vals[:I], want)
    with pytest.raises(L.GsError):
        L.gs_set_wait_limit(-1)


def test_prefix_binning_wait_limit_leaves_valid_lists():
    """The kept-prefix binning's depth sort at look-back limit 0: every tile
    but the first gives up, GS_EW_TIMEOUT is set, the final sort pass
    rewrites its outputs as an identity, and the lists left hold record
    indices only, inside their ranges.  With the default limit the same call
    is exact again."""
    scene = S.uniform_scene(20_000, 3)           # five 4096-record tiles per digit pass
    cam = S.front_camera(256, 256)
    params = P.to_device_params(scene)
    views = dict(P.param_views(params, scene.n))
    fr = P.Frame([cam], scene.n, prefix=True)
    fr.project(views)
    fr.bin_sort()
    fr.render()                                  # the history the kept prefixes are cut by
    fr.bin_sort()
    torch.cuda.synchronize()
    assert fr.check_errors() == 0
    I = int(fr.n_inst.item())
    want_vals, want_ranges = fr.vals[:I].clone(), fr.ranges.clone()
    try:
        L.gs_set_wait_limit(0)
        fr.err.zero_()
        fr.bin_sort()
        torch.cuda.synchronize()
        assert fr.check_errors() & L.GS_EW_TIMEOUT
        n = min(int(fr.n_inst.item()), fr.capacity)
        got = fr.vals[:n]
        assert n == 0 or (int(got.min()) >= 0 and int(got.max()) < scene.n)
        r = fr.ranges.view(-1, 2).long()
        assert bool((r[:, 0] <= r[:, 1]).all()) and int(r[:, 1].max()) <= n
    finally:
        L.gs_set_wait_limit(1 << 20)
    fr.err.zero_()
    fr.bin_sort()
    torch.cuda.synchronize()
    assert fr.check_errors() == 0
    assert torch.equal(fr.ranges, want_ranges) and torch.equal(fr.vals[:I], want_vals)


def test_argument_errors_are_reported():
    cam = S.front_camera(64, 64)
    fr = P.Frame([cam], 8)
    with pytest.raises(L.GsError):
        L.gs_project([cam], 8, None, None, None, None, None, L.GS_F32, fr.splats, L.GS_F32,
                     fr.depth, fr.rect, fr.touched, None, fr.err)
    x = torch.zeros(64, device="cuda")
    with pytest.raises(L.GsError):                            # misaligned quaternions
        L.gs_project([cam], 8, x, x, x[1:], x, x, L.GS_F32, fr.splats, L.GS_F32, fr.depth, fr.rect,
                     fr.touched, None, fr.err)

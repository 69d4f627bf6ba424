"""Parity of the CUDA path with the CPU oracle (needs a GPU).

Discrete results (depth bits, radius, tile rectangles, counts, tile lists,
keys, per-pixel processed counts) must match bit for bit; images within
1e-4 absolute on pixels whose decisions the oracle did not flag as lying
within a rounding margin of the 0.99 / 1/255 / 1e-4 thresholds; gradients
within 1e-3 relative (see tests/_util.py:rel_check).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import GRAD_RTOL, IMG_ATOL, decode_splats, oracle_lists, rel_check

pytestmark = pytest.mark.gpu


def _setup(scene, cams, rgb_dtype=L.GS_F32, sh_dtype=L.GS_F32, keys=True, schedule=None):
    params = P.to_device_params(scene)
    views = P.param_views(params, scene.n)
    if sh_dtype != L.GS_F32:
        views = dict(views)
        views["sh"] = views["sh"].to(torch.bfloat16 if sh_dtype == L.GS_BF16 else torch.float16)
    fr = P.Frame(cams, scene.n, rgb_dtype=rgb_dtype, sh_dtype=sh_dtype, schedule=schedule)
    fr.project(views)
    fr.bin_sort(want_keys=keys)
    fr.render()
    torch.cuda.synchronize()
    return fr, views


CASES = {
    "uniform-10k-256x256": lambda: (S.uniform_scene(10_000, 0), [S.front_camera(256, 256)]),
    # 132 x 132 tiles: many tile rows for the two-pass placement
    "large-view-2112x2100": lambda: (_big(S.uniform_scene(4_000, 9)), [S.front_camera(2112, 2100)]),
    # more than 256 tile columns: the radix-sort binning path
    "wide-view-4160x640": lambda: (_big(S.uniform_scene(3_000, 7)), [S.front_camera(4160, 640)]),
    "ragged-250x190": lambda: (S.uniform_scene(6_000, 5), [S.front_camera(250, 190)]),
    "skewed-20k-200x136": lambda: (S.skewed_scene(20_000, 0), [S.front_camera(200, 136)]),
}


def _big(scene):
    scene.log_scales += 1.5          # large splats: many tiles each
    return scene


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    scene, cams = CASES[request.param]()
    fr, views = _setup(scene, cams)
    refs = []
    for cam in cams:
        kp = O.keypath(cam, scene)
        proj = O.project(cam, scene, kp)
        r = O.render(cam, kp, proj)
        refs.append(dict(kp=kp, proj=proj, r=r))
    return scene, cams, fr, views, refs


def test_discrete_path_bit_exact(case):
    scene, cams, fr, _, refs = case
    kp = refs[0]["kp"]
    n = scene.n
    assert np.array_equal(fr.depth.cpu().numpy().view(np.uint32)[:n][kp["touched"] > 0],
                          kp["depth"].view(np.uint32)[kp["touched"] > 0])
    assert np.array_equal(fr.touched.cpu().numpy()[:n], kp["touched"])
    assert np.array_equal(fr.radius.cpu().numpy()[:n], kp["radius"])
    assert np.array_equal(fr.rect.cpu().numpy().reshape(-1, 4)[:n], kp["rect"])


def test_splat_records(case):
    scene, cams, fr, _, refs = case
    kp, pr = refs[0]["kp"], refs[0]["proj"]
    vis = kp["touched"] > 0
    d = decode_splats(fr.splats.cpu().numpy(), scene.n, L.GS_F32)
    assert np.array_equal(d["u"][vis], kp["mean2d"][vis, 0])
    assert np.array_equal(d["v"][vis], kp["mean2d"][vis, 1])
    for k, c in (("A", 0), ("B", 1), ("C", 2)):
        scale = np.maximum(np.abs(pr["conic"][vis, 0]), np.abs(pr["conic"][vis, 2]))
        assert np.all(np.abs(d[k][vis] - pr["conic"][vis, c]) <= 2e-5 * scale), k
    assert np.allclose(d["opac"][vis], pr["opac"][vis], rtol=2e-5, atol=0)
    assert np.allclose(d["rgb"][vis], pr["rgb"][vis], rtol=0, atol=2e-5)


def test_bin_sort_bit_exact(case):
    scene, cams, fr, _, refs = case
    kp = refs[0]["kp"]
    vals_o, ranges_o = oracle_lists(cams[0], kp)
    I = int(fr.n_inst.item())
    assert I == int(kp["touched"].sum()) == len(vals_o)
    rg = fr.ranges.cpu().numpy().reshape(-1, 2).astype(np.int64)
    cnt = ranges_o[:, 1] - ranges_o[:, 0]
    assert np.array_equal(rg[:, 1] - rg[:, 0], cnt)
    assert np.array_equal(rg[cnt > 0], ranges_o[cnt > 0])       # empty tiles read [0, 0)
    assert np.all(rg[cnt == 0] == 0)
    assert np.array_equal(fr.vals.cpu().numpy()[:I].view(np.uint32), vals_o)
    keys = fr.keys.cpu().numpy()[:I].view(np.uint64)
    tile = np.repeat(np.arange(cams[0].n_tiles, dtype=np.uint64), np.diff(ranges_o, axis=1)[:, 0])
    ref_keys = (tile << np.uint64(32)) | kp["depth"].view(np.uint32)[vals_o].astype(np.uint64)
    assert np.array_equal(keys, ref_keys)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    assert fr.check_errors() == 0


def test_render_forward(case):
    scene, cams, fr, _, refs = case
    r = refs[0]["r"]
    ok = r["flag"] == 0
    assert ok.mean() > 0.98
    img = fr.image(0).cpu().numpy()
    err = np.abs(img - r["img"])[:, ok]
    assert err.max() <= IMG_ATOL, err.max()
    assert np.array_equal(fr.pixel_map(fr.n_proc).cpu().numpy()[ok], r["n_proc"][ok])
    assert np.abs(fr.pixel_map(fr.T_final).cpu().numpy() - r["T_final"])[ok].max() <= IMG_ATOL
    tn = fr.tile_nproc.cpu().numpy()
    npm = fr.pixel_map(fr.n_proc).cpu().numpy()
    cam = cams[0]
    for t in range(cam.n_tiles):
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        assert tn[t] == npm[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16].max()


def _cotangent(cam, flag, seed=3):
    d = S.random_cotangent((3, cam.H, cam.W), seed=seed) * 1e-3
    d[:, flag != 0] = 0.0
    return d


def test_render_backward(case):
    scene, cams, fr, views, refs = case
    cam, ref = cams[0], refs[0]
    dimg = _cotangent(cam, ref["r"]["flag"])
    dimg_t = torch.from_numpy(dimg).cuda().view(-1)
    fr.grad2d.zero_()
    L.gs_render_bwd(fr.cams, fr.ranges, fr.vals, fr.splats, fr.rgb_dtype, None, dimg_t, fr.T_final,
                    fr.n_proc, fr.tile_nproc, fr.grad2d, fr.err)
    g2_gpu = fr.grad2d.cpu().numpy().reshape(-1, 12)[:, :9]
    g2_ref = O.render_bwd(cam, ref["kp"], ref["proj"], dimg.astype(np.float64))
    vis = ref["kp"]["touched"] > 0
    rel_check(g2_gpu[vis], g2_ref[vis], GRAD_RTOL, "grad2d")


def test_project_backward_and_chain(case):
    scene, cams, fr, views, refs = case
    cam, ref = cams[0], refs[0]
    dimg = _cotangent(cam, ref["r"]["flag"], seed=4)
    g2_ref = O.render_bwd(cam, ref["kp"], ref["proj"], dimg.astype(np.float64))
    # projection backward alone, fed the oracle's grad2d
    g2_in = np.zeros((scene.n, 12), np.float32)
    g2_in[:, :9] = g2_ref
    fr.grad2d.copy_(torch.from_numpy(g2_in.ravel()).cuda())
    L.gs_project_bwd(fr.cams, scene.n, views["means"], views["log_scales"], views["quats"],
                     views["opacity_logits"], views["sh"], L.GS_F32, fr.touched, fr.grad2d, fr.dparams)
    gp_ref = O.project_bwd(cam, scene, ref["kp"], g2_in[:, :9].astype(np.float64))
    gp = fr.dparams.cpu().numpy()
    n = scene.n
    for name, (a, b) in dict(means=(0, 3), log_scales=(3, 6), quats=(6, 10), logits=(10, 11),
                             sh=(11, 59)).items():
        rel_check(gp[a * n:b * n].reshape(n, -1), gp_ref[a * n:b * n].reshape(n, -1), GRAD_RTOL,
                  f"project_bwd.{name}")
    # the whole chain on the GPU
    g = fr.backward(views, torch.from_numpy(dimg).cuda().view(-1)).cpu().numpy()
    for name, (a, b) in dict(means=(0, 3), log_scales=(3, 6), quats=(6, 10), logits=(10, 11),
                             sh=(11, 59)).items():
        rel_check(g[a * n:b * n].reshape(n, -1), gp_ref[a * n:b * n].reshape(n, -1),
                  GRAD_RTOL, f"chain.{name}")


def test_l1_loss():
    rng = np.random.default_rng(0)
    n = 3 * 97 * 61
    img = rng.random(n).astype(np.float32)
    tgt = rng.random(n).astype(np.float32)
    tgt[::17] = img[::17]                          # exact ties: zero gradient
    it, tt = torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda()
    loss = torch.zeros(1, device="cuda")
    d = torch.empty_like(it)
    L.gs_l1_loss(n, it, tt, loss, d)
    lo, do = O.l1(img, tgt)
    assert loss.item() == pytest.approx(lo, rel=1e-5)
    assert np.array_equal(np.sign(d.cpu().numpy()), np.sign(do))
    assert np.allclose(d.cpu().numpy(), do, rtol=1e-6, atol=0)


def test_adam_step():
    rng = np.random.default_rng(1)
    N = 1001                                           # 59 N not a multiple of 4
    p0 = rng.normal(size=59 * N).astype(np.float32)
    grads = [rng.normal(size=59 * N).astype(np.float32) for _ in range(3)]
    p = torch.from_numpy(p0).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    shadow = torch.empty(48 * N, dtype=torch.bfloat16, device="cuda")
    lr6 = P.DEFAULT_LR
    lr = np.empty(59 * N)
    lr[:3 * N], lr[3 * N:6 * N], lr[6 * N:10 * N], lr[10 * N:11 * N] = lr6[:4]
    sh_lr = np.where((np.arange(48 * N) % 48) < 3, lr6[4], lr6[5])
    lr[11 * N:] = sh_lr
    po, mo, vo = p0.astype(np.float64), np.zeros(59 * N), np.zeros(59 * N)
    for t, g in enumerate(grads, 1):
        L.gs_adam_step(N, p, torch.from_numpy(g).cuda(), m, v, lr6, 0.9, 0.999, 1e-15, t, shadow, L.GS_BF16)
        po, mo, vo = O.adam(po, g, mo, vo, lr, step=t)
    assert np.allclose(p.cpu().numpy(), po, rtol=0, atol=1e-6)
    assert np.allclose(m.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
    sh_now = p.cpu().numpy()[11 * N:]
    assert torch.equal(shadow.cpu(), torch.from_numpy(sh_now).to(torch.bfloat16))


@pytest.mark.parametrize("sh_dtype", [L.GS_F32, L.GS_BF16])
def test_fused_backward_adam_matches_separate_calls(sh_dtype):
    scene = S.uniform_scene(10_000, 0)
    cam = S.front_camera(256, 256)
    n = scene.n
    params = P.to_device_params(scene)
    views = dict(P.param_views(params, n))
    shadow0 = views["sh"].to(torch.bfloat16) if sh_dtype == L.GS_BF16 else None
    if shadow0 is not None:
        views["sh"] = shadow0
    fr = P.Frame([cam], n, sh_dtype=sh_dtype)
    fr.project(views)
    fr.bin_sort()
    fr.render()
    d = torch.from_numpy(S.random_cotangent((3 * fr.P,), seed=6) * 1e-3).cuda()
    fr.grad2d.zero_()
    L.gs_render_bwd(fr.cams, fr.ranges, fr.vals, fr.splats, fr.rgb_dtype, None, d, fr.T_final, fr.n_proc,
                    fr.tile_nproc, fr.grad2d, fr.err)
    fr.grad2d[:12 * n].view(n, 12)[::7] = 0.0     # Gaussians without a 2D gradient, on both paths
    rng = np.random.default_rng(2)
    m0 = torch.from_numpy(rng.normal(0, 1e-3, 59 * n).astype(np.float32)).cuda()
    v0 = torch.from_numpy(rng.random(59 * n).astype(np.float32) * 1e-6).cuda()
    lr = P.DEFAULT_LR
    # separate calls
    pA, mA, vA = params.clone(), m0.clone(), v0.clone()
    vw = P.param_views(pA, n)
    g = torch.empty(59 * n, device="cuda")
    L.gs_project_bwd([cam], n, vw["means"], vw["log_scales"], vw["quats"], vw["opacity_logits"],
                     shadow0 if shadow0 is not None else vw["sh"], sh_dtype, fr.touched, fr.grad2d, g)
    shA = torch.empty(48 * n, dtype=torch.bfloat16, device="cuda")
    L.gs_adam_step(n, pA, g, mA, vA, lr, 0.9, 0.999, 1e-15, 3, shA, L.GS_BF16)
    # fused
    pB, mB, vB = params.clone(), m0.clone(), v0.clone()
    gB = torch.empty(59 * n, device="cuda")
    shB = torch.empty(48 * n, dtype=torch.bfloat16, device="cuda")
    n_written = int((fr.grad2d[:12 * n].view(n, 12) != 0).any(1).sum())
    assert 0 < n_written < n                      # records with a gradient, and zero ones
    L.gs_project_bwd_adam([cam], n, pB, shadow0, sh_dtype if shadow0 is not None else L.GS_F32, fr.touched,
                          fr.grad2d, mB, vB, lr, 0.9, 0.999, 1e-15, 3, shB, L.GS_BF16, gB)
    torch.cuda.synchronize()
    # the call leaves every record zero (ready for the next reverse pass)
    assert int((fr.grad2d[:12 * n] != 0).sum()) == 0
    # the same backward (two compilations of one source: last-bit differences only)
    assert (g - gB).abs().max() <= 1e-5 * g.abs().max()
    assert torch.allclose(pA, pB, rtol=1e-6, atol=1e-7)
    assert torch.allclose(mA, mB, rtol=1e-6, atol=1e-9)
    assert torch.allclose(vA, vB, rtol=1e-6, atol=1e-12)
    assert (shA.float() - shB.float()).abs().max() <= 2 ** -7 * shA.float().abs().max()

"""Parity at the benchmark's full size (3M skewed Gaussians, 1600x1060), in
the launch configuration bench.py times, on outputs the oracle computes one
by one: every Gaussian's discrete path, every tile's count, the full lists of
sampled tiles, and the image and gradients of the centre 64x64 crop."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import GRAD_RTOL, GROUPS, IMG_ATOL, rel_check, storage_refs, storage_scene

pytestmark = pytest.mark.gpu

WORKLOAD = "skewed-3M-1600x1060"


@pytest.fixture(scope="module")
def full():
    scene, cams = S.make_workload(WORKLOAD, seed=0)
    cam = cams[0]
    kp = O.keypath(cam, scene)
    pr = O.project(cam, scene, kp)
    return scene, cam, kp, pr


def _trainer(scene, cams, mode, dtype):
    tgt = torch.from_numpy(S.random_image(cams[0].W, cams[0].H, seed=1).ravel()).cuda()
    return P.Trainer(cams, P.to_device_params(scene), scene.n, tgt, rgb_dtype=dtype,
                     sh_storage=dtype, schedule=P.Schedule(mode=mode))


def _crop(cam, size=64):
    x0, y0 = (cam.W - size) // 2 // 16 * 16, (cam.H - size) // 2 // 16 * 16
    return x0, y0, x0 + size, y0 + size


def test_fullsize_fp32_count_path(full):
    scene, cam, kp, pr = full
    tr = _trainer(scene, [cam], "count", L.GS_F32)
    f = tr.frame
    pk = tr.params_for_kernels()
    f.forward(pk)
    torch.cuda.synchronize()
    assert f.check_errors() == 0
    # every Gaussian's discrete path
    assert np.array_equal(f.touched.cpu().numpy(), kp["touched"])
    assert np.array_equal(f.rect.cpu().numpy().reshape(-1, 4), kp["rect"])
    # every tile's full count; the kept prefixes of sampled tiles (the
    # training step bins with gs_bin_sort_prefix)
    counts = O.tile_counts(cam, kp)
    assert np.array_equal(f.tile_count.cpu().numpy().astype(np.int64), counts)
    rg = f.ranges.cpu().numpy().reshape(-1, 2).astype(np.int64)
    kept = rg[:, 1] - rg[:, 0]
    assert np.all(kept <= counts) and int(f.n_inst.item()) == int(kept.sum())
    vals = f.vals.cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(0)
    sample = set(rng.choice(cam.n_tiles, 8, replace=False).tolist())
    sample |= {int(np.argmax(counts)), 0, cam.n_tiles - 1, cam.tiles_x - 1}
    for t in sorted(sample):
        ids = O.tile_list(kp, t % cam.tiles_x, t // cam.tiles_x)[:kept[t]]
        assert np.array_equal(vals[rg[t, 0]:rg[t, 1]], ids), t
    # the centre crop: image and gradients
    win = _crop(cam)
    r = O.render(cam, kp, pr, window=win)
    x0, y0, x1, y1 = win
    ok = r["flag"][y0:y1, x0:x1] == 0
    assert ok.mean() > 0.95
    img = f.image(0).cpu().numpy()[:, y0:y1, x0:x1]
    assert np.abs(img - r["img"][:, y0:y1, x0:x1])[:, ok].max() <= IMG_ATOL
    npm = f.pixel_map(f.n_proc).cpu().numpy()[y0:y1, x0:x1]
    assert np.array_equal(npm[ok], r["n_proc"][y0:y1, x0:x1][ok])
    d = np.zeros((3, cam.H, cam.W), np.float32)
    dc = S.random_cotangent((3, y1 - y0, x1 - x0), seed=8) * 1e-3
    dc[:, ~ok] = 0.0
    d[:, y0:y1, x0:x1] = dc
    g = f.backward(pk, torch.from_numpy(d.ravel()).cuda()).cpu().numpy()
    g2 = O.render_bwd(cam, kp, pr, d.astype(np.float64), window=win)
    gref = O.project_bwd(cam, scene, kp, g2)
    n = scene.n
    hit = np.abs(g2).sum(1) > 0
    assert hit.sum() > 100
    for name, (a, b) in dict(means=(0, 3), log_scales=(3, 6), quats=(6, 10), logits=(10, 11),
                             sh=(11, 59)).items():
        gg = g[a * n:b * n].reshape(n, -1)
        gr = gref[a * n:b * n].reshape(n, -1)
        rel_check(gg[hit], gr[hit], GRAD_RTOL, name)
        assert np.all(gg[~hit] == 0.0), name


def _crop_gaussians(cam, kp, win):
    """Visible Gaussians whose tile rectangle meets the crop's tiles."""
    x0, y0, x1, y1 = (v // 16 for v in win)
    r = kp["rect"]
    return np.flatnonzero((kp["touched"] > 0) & (r[:, 0] < x1) & (r[:, 2] > x0) & (r[:, 1] < y1) & (r[:, 3] > y0))


def test_fullsize_bf16_learned_path(full):
    """The benchmark's precision path at full size: BF16 SH and colours,
    kept-prefix binning, the learned order a few steps in.  The centre crop's
    image, reverse pass, projection backward and fused backward + Adam
    against the oracle of the storage path (same rounded SH, colours rounded
    to BF16; tests/test_gpu_half_grad.py)."""
    scene, cam, kp, _ = full
    win = _crop(cam)
    sc = storage_scene(scene, [cam], L.GS_BF16, only=_crop_gaussians(cam, kp, win))
    tr = _trainer(sc, [cam], "learned", L.GS_BF16)
    f = tr.frame
    for _ in range(3):                      # the benchmark's configuration, a few steps in
        f.forward(tr.params_for_kernels(), timing=True)
        f.l1(tr.targets)
        f.render_bwd(f.dimg, timing=True)
        f.train_scheduler()
    f.use_learned = True                    # the reverse pass in the learned order
    pk = tr.params_for_kernels()
    f.forward(pk, timing=True)
    torch.cuda.synchronize()
    assert f.check_errors() == 0
    ref = storage_refs(sc, [cam], L.GS_BF16, window=win)[0]
    r, kp16, pr16 = ref["r"], ref["kp"], ref["proj"]
    x0, y0, x1, y1 = win
    ok = r["flag"][y0:y1, x0:x1] == 0
    print(f"\nflagged crop pixels: {1 - ok.mean():.2%}")
    assert ok.mean() > 0.95
    img = f.image(0).cpu().numpy()[:, y0:y1, x0:x1]
    assert np.abs(img - r["img"][:, y0:y1, x0:x1])[:, ok].max() <= IMG_ATOL
    # gradients of a cotangent on the crop
    d = np.zeros((3, cam.H, cam.W), np.float32)
    dc = S.random_cotangent((3, y1 - y0, x1 - x0), seed=8) * 1e-3
    dc[:, ~ok] = 0.0
    d[:, y0:y1, x0:x1] = dc
    d_t = torch.from_numpy(d.ravel()).cuda()
    g2 = O.render_bwd(cam, kp16, pr16, d.astype(np.float64), window=win)
    gref = O.project_bwd(cam, sc, kp16, g2)
    n = sc.n
    hit = np.abs(g2).sum(1) > 0
    assert hit.sum() > 100
    g = f.backward(pk, d_t).cpu().numpy()
    # the fused call the training step makes (BF16 shadow read and rewritten)
    f.grad2d.zero_()
    L.gs_render_bwd(f.cams, f.ranges, f.vals, f.splats, f.rgb_dtype, None, d_t, f.T_final, f.n_proc,
                    f.tile_nproc, f.grad2d, f.err)
    gB = torch.empty(59 * n, device="cuda")
    L.gs_project_bwd_adam([cam], n, tr.p, tr.sh_shadow, L.GS_BF16, f.touched, f.grad2d, tr.m, tr.v,
                          tr.lr, P.ADAM_B1, P.ADAM_B2, P.ADAM_EPS, 1, tr.sh_shadow, L.GS_BF16, gB)
    gb = gB.cpu().numpy()
    for name, (a, b) in GROUPS.items():
        gr = gref[a * n:b * n].reshape(n, -1)
        for what, got in (("chain", g), ("fused", gb)):
            gg = got[a * n:b * n].reshape(n, -1)
            rel_check(gg[hit], gr[hit], GRAD_RTOL, f"{what}.{name}")
            assert np.all(gg[~hit] == 0.0), f"{what}.{name}"

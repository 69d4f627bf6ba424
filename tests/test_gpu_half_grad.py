"""Gradients of the 16-bit storage path against the oracle (needs a GPU).

SH coefficients are read as BF16 or FP16 and record colours stored in the
same format; blending, conics and every gradient stay FP32.  The oracle of
this path reads the same rounded SH, evaluates the colour in FP64 and
rounds it to the storage format (O.round_storage, pinned on the CPU), then
blends and differentiates in FP64.  Scenes are prepared so that no visible
colour lies within FP32 error of a rounding point (tests/_util.py
storage_scene): both sides then hold the same 16-bit colours, and the FP32
tolerances apply unchanged -- images within 1e-4 on unflagged pixels,
gradients within 1e-3 relative.

Each call of the precision path is covered: gs_render_bwd on 16-bit records
(a5), gs_project_bwd on 16-bit SH (a6), the fused gs_project_bwd_adam with
a 16-bit SH shadow (a6 + a7), and one whole Trainer.step.  Against the
oracle of the FP32 scene (unrounded SH and colours) the error of the storage
itself is printed per parameter group."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import (GRAD_RTOL, GROUPS, IMG_ATOL, STORAGE_KIND, blending_at_flagged, rel_check,
                         rel_errors, storage_refs, storage_scene)

pytestmark = pytest.mark.gpu

TDT = {L.GS_BF16: torch.bfloat16, L.GS_F16: torch.float16}

CASES = {
    "uniform-10k-256x256": lambda: (S.uniform_scene(10_000, 0), S.front_camera(256, 256)),
    "skewed-20k-200x136": lambda: (S.skewed_scene(20_000, 0), S.front_camera(200, 136)),
}


def _views16(sc, dtype):
    params = P.to_device_params(sc)
    views = dict(P.param_views(params, sc.n))
    views["sh"] = views["sh"].to(TDT[dtype])       # exact: sc's SH are representable
    return params, views


def _frame(sc, cam, dtype):
    params, views = _views16(sc, dtype)
    fr = P.Frame([cam], sc.n, rgb_dtype=dtype, sh_dtype=dtype)
    fr.project(views)
    fr.bin_sort()
    fr.render()
    torch.cuda.synchronize()
    return fr, params, views


def _cotangent(cam, flag, seed):
    d = S.random_cotangent((3, cam.H, cam.W), seed=seed) * 1e-3
    d[:, flag != 0] = 0.0
    return d


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", [L.GS_BF16, L.GS_F16], ids=["bf16", "f16"])
def test_half_storage_forward_and_gradients_match_oracle(case, dtype):
    scene, cam = CASES[case]()
    sc = storage_scene(scene, [cam], dtype)
    ref = storage_refs(sc, [cam], dtype)[0]
    kp, pr, r = ref["kp"], ref["proj"], ref["r"]
    fr, params, views = _frame(sc, cam, dtype)
    assert fr.check_errors() == 0
    n = sc.n
    ok = r["flag"] == 0
    print(f"\n{case} {STORAGE_KIND[dtype]}: flagged pixels {1 - ok.mean():.3%}")
    assert ok.mean() > 0.98
    # forward: the same 16-bit colours on both sides, so the FP32 bound holds
    img = fr.image(0).cpu().numpy()
    assert np.abs(img - r["img"])[:, ok].max() <= IMG_ATOL
    assert np.array_equal(fr.pixel_map(fr.n_proc).cpu().numpy()[ok], r["n_proc"][ok])
    # a5 on 16-bit records
    dimg = _cotangent(cam, r["flag"], seed=3)
    fr.grad2d.zero_()
    L.gs_render_bwd(fr.cams, fr.ranges, fr.vals, fr.splats, fr.rgb_dtype, None,
                    torch.from_numpy(dimg).cuda().view(-1), fr.T_final, fr.n_proc, fr.tile_nproc,
                    fr.grad2d, fr.err)
    g2_ref = O.render_bwd(cam, kp, pr, dimg.astype(np.float64))
    vis = kp["touched"] > 0
    rel_check(fr.grad2d.cpu().numpy().reshape(-1, 12)[:n, :9][vis], g2_ref[vis], GRAD_RTOL, "grad2d")
    # a6 on 16-bit SH, fed the oracle's 2D gradient
    g2_in = np.zeros((n, 12), np.float32)
    g2_in[:, :9] = g2_ref
    fr.grad2d.copy_(torch.from_numpy(g2_in.ravel()).cuda())
    L.gs_project_bwd(fr.cams, n, views["means"], views["log_scales"], views["quats"],
                     views["opacity_logits"], views["sh"], dtype, fr.touched, fr.grad2d, fr.dparams)
    gp_ref = O.project_bwd(cam, sc, kp, g2_in[:, :9].astype(np.float64))
    gp = fr.dparams.cpu().numpy()
    for name, (a, b) in GROUPS.items():
        rel_check(gp[a * n:b * n].reshape(n, -1), gp_ref[a * n:b * n].reshape(n, -1), GRAD_RTOL,
                  f"project_bwd.{name}")
    # the chain a5 -> a6
    d_t = torch.from_numpy(dimg).cuda().view(-1)
    g = fr.backward(views, d_t).cpu().numpy()
    chain_ref = O.project_bwd(cam, sc, kp, g2_ref)
    for name, (a, b) in GROUPS.items():
        rel_check(g[a * n:b * n].reshape(n, -1), chain_ref[a * n:b * n].reshape(n, -1), GRAD_RTOL,
                  f"chain.{name}")
    # a6 + a7 fused, the 16-bit shadow read by the backward and rewritten by Adam
    fr.grad2d.zero_()
    L.gs_render_bwd(fr.cams, fr.ranges, fr.vals, fr.splats, fr.rgb_dtype, None, d_t, fr.T_final,
                    fr.n_proc, fr.tile_nproc, fr.grad2d, fr.err)
    p = params.clone()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    shadow = views["sh"].clone()
    gB = torch.empty(59 * n, device="cuda")
    L.gs_project_bwd_adam([cam], n, p, shadow, dtype, fr.touched, fr.grad2d, m, v, P.DEFAULT_LR,
                          P.ADAM_B1, P.ADAM_B2, P.ADAM_EPS, 1, shadow, dtype, gB)
    torch.cuda.synchronize()
    gb = gB.cpu().numpy()
    for name, (a, b) in GROUPS.items():
        rel_check(gb[a * n:b * n].reshape(n, -1), chain_ref[a * n:b * n].reshape(n, -1), GRAD_RTOL,
                  f"fused.{name}")
    _check_adam_step(p, m, shadow, sc.flat().astype(np.float64), chain_ref, n, dtype)
    # the error of the storage itself: against the FP64 oracle of the FP32 scene
    _report_accuracy(scene, cam, dtype, case)


def _lr_per_entry(n):
    lr6 = P.DEFAULT_LR
    lr = np.empty(59 * n)
    lr[:3 * n], lr[3 * n:6 * n], lr[6 * n:10 * n], lr[10 * n:11 * n] = lr6[:4]
    lr[11 * n:] = np.where((np.arange(48 * n) % 48) < 3, lr6[4], lr6[5])
    return lr


def _check_adam_step(p, m, shadow, p0, grads, n, dtype, keep=None):
    """First Adam step from zero moments: m = (1 - b1) g; p moves by lr g /
    (|g| + eps) where the gradient is resolved, by at most lr everywhere; the
    shadow is the storage rounding of the updated SH."""
    keep = np.ones(n, bool) if keep is None else keep
    lr = _lr_per_entry(n)
    g_gpu = m.cpu().numpy().astype(np.float64) / (1.0 - P.ADAM_B1)
    pg_all = p.cpu().numpy().astype(np.float64)
    p_ref, _, _ = O.adam(p0, grads, np.zeros(59 * n), np.zeros(59 * n), lr, step=1)
    for name, (a, b) in GROUPS.items():
        w = b - a
        sl = lambda x: x[a * n:b * n].reshape(n, w)[keep]
        rel_check(sl(g_gpu), sl(grads), GRAD_RTOL, f"adam.m.{name}")
        pg, pr, p0g, lrg, gr = sl(pg_all), sl(p_ref), sl(p0), sl(lr), sl(grads)
        sig = np.abs(gr) >= 1e-2 * np.abs(gr).max(axis=0, keepdims=True)
        assert np.all(np.abs(pg - pr)[sig] <= 4e-7 * np.maximum(1.0, np.abs(pr[sig])) + 1e-4 * lrg[sig]), name
        assert np.all(np.abs(pg - p0g) <= lrg * (1 + 1e-5) + 4e-7 * np.maximum(1.0, np.abs(p0g))), name
    sh_new = pg_all[11 * n:]
    want = O.round_storage(sh_new.astype(np.float32).astype(np.float64), STORAGE_KIND[dtype])
    assert np.array_equal(shadow.float().cpu().numpy().ravel().astype(np.float64), want)


def _report_accuracy(scene, cam, dtype, case):
    """Image and gradient error of the 16-bit storage path on the unprepared
    FP32 scene against the FP64 oracle of that scene (unrounded SH and
    colours).  Printed per result; bounded only loosely (the rounding of
    colours to 8 or 11 significant bits)."""
    n = scene.n
    params = P.to_device_params(scene)
    views = dict(P.param_views(params, n))
    views["sh"] = views["sh"].to(TDT[dtype])
    fr = P.Frame([cam], n, rgb_dtype=dtype, sh_dtype=dtype)
    fr.project(views)
    fr.bin_sort()
    fr.render()
    r = O.forward(cam, scene)
    ok = r["flag"] == 0
    img_err = np.abs(fr.image(0).cpu().numpy() - r["img"])[:, ok]
    dimg = _cotangent(cam, r["flag"], seed=3)
    g = fr.backward(views, torch.from_numpy(dimg).cuda().view(-1)).cpu().numpy()
    gref = O.project_bwd(cam, scene, r["kp"], O.render_bwd(cam, r["kp"], r["proj"], dimg.astype(np.float64)))
    vis = r["kp"]["touched"] > 0
    line = [f"image max {img_err.max():.2e} mean {img_err.mean():.2e}"]
    for name, (a, b) in GROUPS.items():
        mx, med = rel_errors(g[a * n:b * n].reshape(n, -1)[vis], gref[a * n:b * n].reshape(n, -1)[vis])
        line.append(f"{name} {mx:.2e}/{med:.2e}")
        assert mx < 2.0 ** -4, name
    print(f"{case} {STORAGE_KIND[dtype]} storage vs FP64 oracle of the FP32 scene "
          f"(gradient: max-norm relative / median relative): " + ", ".join(line))


def test_bf16_training_step_matches_oracle():
    """One whole Trainer.step with BF16 SH and colours (kept-prefix binning,
    count order, fused projection backward + Adam) against the oracle chain of
    the storage path: forward with rounded colours, L1 over the view, reverse
    blending, projection backward, Adam on the FP32 master copy.  Then the
    same step again from the same state, binned from the first step's
    history."""
    dtype = L.GS_BF16
    scene = S.uniform_scene(1500, 3)
    cam = S.front_camera(112, 72)
    sc = storage_scene(scene, [cam], dtype)
    ref = storage_refs(sc, [cam], dtype)[0]
    r = ref["r"]
    n = sc.n
    tgt = S.random_image(cam.W, cam.H, seed=20).astype(np.float64)
    close = np.abs(r["img"] - tgt) < 0.02             # keep the sign of the L1 gradient clear
    tgt[close] = np.where(r["img"][close] < 0.5, r["img"][close] + 0.05, r["img"][close] - 0.05)
    tgt = tgt.astype(np.float32)
    _, d = O.l1(r["img"], tgt.astype(np.float64))
    grads = O.project_bwd(cam, sc, ref["kp"], O.render_bwd(cam, ref["kp"], ref["proj"], d))
    keep = ~blending_at_flagged(cam, ref["kp"], ref["proj"], r["flag"])
    print(f"\nflagged pixels {np.mean(r['flag'] != 0):.3%}; Gaussians compared {keep.mean():.1%}")
    assert keep.mean() >= 0.9
    p0 = sc.flat().astype(np.float64)
    tr = P.Trainer([cam], P.to_device_params(sc), n, torch.from_numpy(tgt.ravel()).cuda(), rgb_dtype=dtype,
                   sh_storage=dtype, schedule=P.Schedule("count"))
    for _ in range(2):
        tr.step()
        torch.cuda.synchronize()
        assert tr.frame.check_errors() == 0
        _check_adam_step(tr.p, tr.m, tr.sh_shadow, p0, grads, n, dtype, keep)
        tr.p.copy_(torch.from_numpy(sc.flat()).cuda())
        tr.sh_shadow.copy_(tr.views["sh"].to(torch.bfloat16))
        tr.m.zero_()
        tr.v.zero_()
        tr.t = 0

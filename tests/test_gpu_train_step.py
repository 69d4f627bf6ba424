"""One whole training step through Trainer.step against the oracle chain:
projection, binning, blending, L1 over every view's pixels, backward
blending, projection backward and Adam.  One view takes the fused projection
backward + Adam kernel, two views the separate calls.

Pixels the oracle flags (a discrete decision within rounding of a threshold)
may legitimately differ; every Gaussian that blends at one of them is left
out of the comparison (at least 90% of the Gaussians stay in).  The target
is pushed away from the oracle image where they are close, so the sign of
the L1 gradient is the same on both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import GRAD_RTOL, blending_at_flagged, rel_check

pytestmark = pytest.mark.gpu

GROUPS = dict(means=(0, 3), log_scales=(3, 6), quats=(6, 10), logits=(10, 11), sh=(11, 59))


def _lr_per_entry(n):
    lr6 = P.DEFAULT_LR
    lr = np.empty(59 * n)
    lr[:3 * n], lr[3 * n:6 * n], lr[6 * n:10 * n], lr[10 * n:11 * n] = lr6[:4]
    lr[11 * n:] = np.where((np.arange(48 * n) % 48) < 3, lr6[4], lr6[5])
    return lr


def _oracle_step(scene, cams, seed):
    """Targets, the oracle gradient of the mean L1 over all views, and the
    Gaussians near a flagged pixel."""
    n = scene.n
    n_total = sum(3 * c.W * c.H for c in cams)
    grads = np.zeros(59 * n)
    excluded = np.zeros(n, bool)
    tgts = []
    for v, cam in enumerate(cams):
        r = O.forward(cam, scene)
        img = r["img"]
        tgt = S.random_image(cam.W, cam.H, seed=seed + v).astype(np.float64)
        close = np.abs(img - tgt) < 0.02
        tgt[close] = np.where(img[close] < 0.5, img[close] + 0.05, img[close] - 0.05)
        tgt = tgt.astype(np.float32)
        tgts.append(tgt)
        _, d = O.l1(img, tgt.astype(np.float64))
        d *= d.size / n_total                  # the loss is the mean over every view's pixels
        g2 = O.render_bwd(cam, r["kp"], r["proj"], d)
        grads += O.project_bwd(cam, scene, r["kp"], g2)
        excluded |= blending_at_flagged(cam, r["kp"], r["proj"], r["flag"])
    return tgts, grads, excluded


def _check(tr, scene, p0, grads, excluded, b1=P.ADAM_B1):
    n = scene.n
    keep = ~excluded
    print(f"\nGaussians compared: {keep.mean():.1%}")
    assert keep.mean() >= 0.9
    m = tr.m.cpu().numpy().astype(np.float64)
    p = tr.p.cpu().numpy().astype(np.float64)
    g_gpu = m / (1.0 - b1)                    # first step from m = 0: m = (1 - b1) g
    p_ref, _, _ = O.adam(p0, grads, np.zeros(59 * n), np.zeros(59 * n), _lr_per_entry(n), step=1)
    lr = _lr_per_entry(n)
    for name, (a, b) in GROUPS.items():
        w = b - a
        gg = g_gpu[a * n:b * n].reshape(n, w)[keep]
        gr = grads[a * n:b * n].reshape(n, w)[keep]
        rel_check(gg, gr, GRAD_RTOL, name)
        pg = p[a * n:b * n].reshape(n, w)[keep]
        pr = p_ref[a * n:b * n].reshape(n, w)[keep]
        p0g = p0[a * n:b * n].reshape(n, w)[keep]
        lrg = lr[a * n:b * n].reshape(n, w)[keep]
        # resolved gradients: the step lr * g / |g| of the oracle, to FP32 rounding
        sig = np.abs(gr) >= 1e-2 * np.abs(gr).max(axis=0, keepdims=True)
        assert np.all(np.abs(pg - pr)[sig] <= 4e-7 * np.maximum(1.0, np.abs(pr[sig])) + 1e-4 * lrg[sig]), name
        # every entry moves by at most lr
        assert np.all(np.abs(pg - p0g) <= lrg * (1 + 1e-5) + 4e-7 * np.maximum(1.0, np.abs(p0g))), name


def _trainer(scene, cams, tgts):
    tflat = torch.from_numpy(np.concatenate([t.ravel() for t in tgts])).cuda()
    return P.Trainer(cams, P.to_device_params(scene), scene.n, tflat, rgb_dtype=L.GS_F32,
                     sh_storage=L.GS_F32, schedule=P.Schedule("count"))


@pytest.mark.parametrize("views", [1, 2])
def test_training_step_matches_oracle(views):
    scene = S.uniform_scene(1500, 3)
    if views == 1:
        cams = [S.front_camera(112, 72)]
    else:
        cams = S.ring_cameras(2, [(112, 72), (80, 64)])
    tgts, grads, excluded = _oracle_step(scene, cams, seed=20)
    p0 = scene.flat().astype(np.float64)
    tr = _trainer(scene, cams, tgts)
    tr.step()
    torch.cuda.synchronize()
    assert tr.frame.check_errors() == 0
    _check(tr, scene, p0, grads, excluded)
    # the same step again from the same state: now binned with the kept
    # prefixes the first step's counts allow (history limits, repair)
    tr.p.copy_(torch.from_numpy(scene.flat()).cuda())
    tr.m.zero_()
    tr.v.zero_()
    tr.t = 0
    tr.step()
    torch.cuda.synchronize()
    assert tr.frame.check_errors() == 0
    _check(tr, scene, p0, grads, excluded)


def test_bf16_training_step_updates_master_and_shadow():
    """BF16 SH storage: the fused kernel updates the FP32 master copy and
    writes its BF16 rounding to the shadow the next forward reads; the update
    equals the separate backward + Adam calls."""
    scene = S.uniform_scene(1500, 3)
    cams = [S.front_camera(112, 72)]
    tgt = torch.from_numpy(S.random_image(112, 72, seed=20).ravel()).cuda()
    trs = [P.Trainer(cams, P.to_device_params(scene), scene.n, tgt, rgb_dtype=L.GS_BF16,
                     sh_storage=L.GS_BF16, schedule=P.Schedule("count")) for _ in range(2)]
    trs[0].step()
    # the second trainer: the same step with the separate calls
    tr = trs[1]
    f = tr.frame
    pk = tr.params_for_kernels()
    f.project(pk)
    f.bin_sort()
    f.render()
    f.l1(tr.targets)
    f.grad2d.zero_()
    L.gs_render_bwd(f.cams, f.ranges, f.vals, f.splats, f.rgb_dtype, None, f.dimg, f.T_final, f.n_proc,
                    f.tile_nproc, f.grad2d, f.err)
    L.gs_project_bwd(f.cams, tr.N, pk["means"], pk["log_scales"], pk["quats"], pk["opacity_logits"],
                     tr.sh_shadow, L.GS_BF16, f.touched, f.grad2d, f.dparams)
    L.gs_adam_step(tr.N, tr.p, f.dparams, tr.m, tr.v, tr.lr, P.ADAM_B1, P.ADAM_B2, P.ADAM_EPS, 1,
                   tr.sh_shadow, L.GS_BF16)
    torch.cuda.synchronize()
    a, b = trs
    assert a.frame.check_errors() == 0 and b.frame.check_errors() == 0
    n = scene.n
    # the same gradients up to the rounding of two compilations (m = (1 - b1) g)
    assert (a.m - b.m).abs().max() <= 1e-5 * b.m.abs().max()
    sh_a = a.p[11 * n:]
    assert torch.equal(a.sh_shadow.view(-1), sh_a.to(torch.bfloat16))
    moved = (a.p - torch.from_numpy(scene.flat()).cuda()).abs()
    assert moved.max() > 0


def test_next_step_reuses_the_records_the_fused_call_zeroed():
    """One view: the fused backward + Adam leaves the 2D-gradient records all
    zero, so the next step's reverse pass adds into them without a memset;
    two steps that way equal two steps with the records zeroed explicitly."""
    scene = S.uniform_scene(1500, 4)
    cams = [S.front_camera(112, 72)]
    tgt = torch.from_numpy(S.random_image(112, 72, seed=21).ravel()).cuda()
    trs = [P.Trainer(cams, P.to_device_params(scene), scene.n, tgt, rgb_dtype=L.GS_BF16,
                     sh_storage=L.GS_BF16, schedule=P.Schedule("count")) for _ in range(2)]
    n = scene.n
    for k, tr in enumerate(trs):
        tr.step()
        torch.cuda.synchronize()
        assert tr.frame.grad2d_zero
        assert int((tr.frame.grad2d[:12 * n] != 0).sum()) == 0
        if k == 1:
            tr.frame.grad2d_zero = False          # the second trainer zeroes again before its reverse pass
        tr.step()
    torch.cuda.synchronize()
    a, b = trs
    assert a.frame.check_errors() == 0 and b.frame.check_errors() == 0
    # equal up to the order of the reverse pass's atomic additions
    assert (a.m - b.m).abs().max() <= 1e-5 * b.m.abs().max()
    assert (a.p - b.p).abs().max() <= 1e-5 * b.p.abs().max()


def test_target_of_the_wrong_size_is_refused():
    """The L1 target covers every view's pixels; a target for one view of a
    two-view batch is refused on the host, before the L1 kernel runs."""
    scene = S.uniform_scene(500, 1)
    cams = S.ring_cameras(2, [(64, 48), (48, 32)])
    one_view = torch.zeros(3 * 64 * 48, device="cuda")
    with pytest.raises(ValueError):
        P.Trainer(cams, P.to_device_params(scene), scene.n, one_view)
    both = torch.zeros(3 * (64 * 48 + 48 * 32), device="cuda")
    tr = P.Trainer(cams, P.to_device_params(scene), scene.n, both)
    with pytest.raises(ValueError):
        tr.step(targets=one_view)

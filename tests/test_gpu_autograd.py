"""RasterizeGaussians, the torch.autograd.Function over the CUDA path (needs
a GPU), on 1024-Gaussian subsets of the 3M-Gaussian 1600x1060 scene.

Two checks of its backward, for FP32 storage and for BF16 SH and colours:

- against the oracle gradient (FP64 reverse mode of the same forward; for
  BF16 the oracle of the storage path, tests/test_gpu_half_grad.py), within
  1e-3 relative; the BF16 SH gradient comes back in BF16, the dtype of its
  input, so its bound adds that rounding (2^-8 relative);
- against central differences of the GPU forward itself: <dL/dp, v> for
  random directions v on random groups of visible Gaussians, with
  L = sum(dimg * image).  The forward is piecewise smooth: its discrete
  decisions (tile rectangles, the alpha skip and clamp, the transmittance
  stop, the colour clamp) must not change between p - v and p + v.  Pixels
  with a blending decision within 10% of its threshold carry no upstream
  gradient, directions whose tile rectangles change (the oracle's FP32 key
  path, bit-exact with the GPU's) are drawn again, Gaussians with a colour
  near the clamp are not perturbed (with BF16 colours, which are piecewise
  constant in the view direction, neither are means or SH), and a mean moves along the viewing axis
  only when no Gaussian sharing a tile with it lies within 20 steps in depth
  (the depth order of a tile list must not change either).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import GRAD_RTOL, GROUPS, rel_check, storage_refs, storage_scene

pytestmark = pytest.mark.gpu

N_SUB = 1024
FD_MARGIN = 0.1           # flag margin of the FD check (alpha and transmittance, relative)
FD_RTOL, FD_ATOL = 5e-3, 1e-4   # FP32 rounding of the two renders limits the absolute part
# per-group perturbation scale (about 0.3% of a Gaussian's size for the
# means, 5e-4 of the unit for log-scales, quaternions, logits, SH): alpha
# moves by well under the flag margin, and few tile rectangles change
STEP = dict(means=5e-5, log_scales=5e-4, quats=5e-4, logits=5e-4, sh=5e-4)
N_DIR, N_MOVED, MAX_TRIES = 6, 12, 30
TDT = {L.GS_F32: torch.float32, L.GS_BF16: torch.bfloat16}


@pytest.fixture(scope="module")
def subsets():
    scene, cams = S.make_workload("skewed-3M-1600x1060", seed=0)
    rng = np.random.default_rng(5)
    out = [scene.subset(np.sort(rng.choice(scene.n, N_SUB, replace=False))) for _ in range(2)]
    return out, cams[0]


def _leaves(sc, dtype):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    return [t(sc.means), t(sc.log_scales), t(sc.quats), t(sc.opacity_logits),
            t(sc.sh).to(TDT[dtype])]


def _loss(leaves, cam, dtype, dimg_t):
    with torch.no_grad():
        img = P.RasterizeGaussians.apply(*leaves, cam, dtype)
    return float((img.double() * dimg_t).sum())


def _refs(sc, cam, dtype):
    if dtype == L.GS_F32:
        kp = O.keypath(cam, sc)
        pr = O.project(cam, sc, kp)
        return kp, pr
    ref = storage_refs(sc, [cam], dtype)[0]
    return ref["kp"], ref["proj"]


@pytest.mark.parametrize("dtype", [L.GS_F32, L.GS_BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("which", [0, 1])
def test_autograd_function_against_oracle_and_finite_differences(subsets, dtype, which):
    subs, cam = subsets
    sc = subs[which]
    if dtype != L.GS_F32:
        sc = storage_scene(sc, [cam], dtype)
    n = sc.n
    kp, pr = _refs(sc, cam, dtype)
    r = O.render(cam, kp, pr, margin_alpha=FD_MARGIN, margin_T=FD_MARGIN)
    dimg = S.random_cotangent((3, cam.H, cam.W), seed=30 + which)
    dimg[:, r["flag"] != 0] = 0.0
    dimg_t = torch.from_numpy(dimg).cuda()
    # backward through autograd
    leaves = [x.requires_grad_(True) for x in _leaves(sc, dtype)]
    img = P.RasterizeGaussians.apply(*leaves, cam, dtype)
    assert img.shape == (3, cam.H, cam.W) and img.dtype == torch.float32
    grads = torch.autograd.grad(img, leaves, grad_outputs=dimg_t)
    assert grads[4].dtype == TDT[dtype] and grads[4].shape == (n, 16, 3)
    g = {name: grads[k].double().cpu().numpy().reshape(n, -1) for k, name in enumerate(GROUPS)}
    # against the oracle gradient
    gref = O.project_bwd(cam, sc, kp, O.render_bwd(cam, kp, pr, dimg.astype(np.float64)))
    gref = {name: gref[a * n:b * n].reshape(n, -1) for name, (a, b) in GROUPS.items()}
    vis = kp["touched"] > 0
    print(f"\n{vis.sum()} of {n} Gaussians visible; flagged pixels {np.mean(r['flag'] != 0):.3%}")
    assert vis.sum() > 200
    for name in GROUPS:
        if name == "sh" and dtype != L.GS_F32:
            # returned in BF16: the FP32 gradient rounded once more
            gr, gg = gref[name][vis], g[name][vis]
            scale = np.abs(gr).max(axis=0, keepdims=True)
            assert np.all(np.abs(gg - gr) <= 2.0 ** -8 * np.abs(gr) + GRAD_RTOL * scale), name
            continue
        rel_check(g[name][vis], gref[name][vis], GRAD_RTOL, f"autograd.{name}")
    # central differences of the GPU forward
    rng = np.random.default_rng(40 + which)
    smooth = vis & (np.abs(pr["rgb_pre"]).min(axis=1) > 0.02)
    # depth gap to the nearest visible Gaussian whose tile rectangle overlaps
    rc, dep = kp["rect"], kp["depth"].astype(np.float64)
    over = ((rc[:, None, 0] < rc[None, :, 2]) & (rc[None, :, 0] < rc[:, None, 2]) &
            (rc[:, None, 1] < rc[None, :, 3]) & (rc[None, :, 1] < rc[:, None, 3]) & vis[:, None] & vis[None, :])
    np.fill_diagonal(over, False)
    gap = np.where(over, np.abs(dep[:, None] - dep[None, :]), np.inf).min(axis=1)
    depth_free = gap > 20 * 4 * STEP["means"]
    axis = np.asarray(cam.R, np.float64)[2]             # camera viewing axis in world space
    # 16-bit colours are piecewise constant in the view direction (a mean's
    # move crosses their rounding steps), so with BF16 only scales,
    # rotations and opacities are perturbed
    perturbed = (["means", "log_scales", "quats", "logits", "sh"] if dtype == L.GS_F32
                 else ["log_scales", "quats", "logits"])
    done = tries = 0
    while done < N_DIR and tries < MAX_TRIES:
        tries += 1
        ids = rng.choice(np.flatnonzero(smooth), N_MOVED, replace=False)
        v = {name: np.zeros_like(g[name]) for name in GROUPS}
        for name in perturbed:
            v[name][ids] = rng.normal(0.0, 1.0, (len(ids), v[name].shape[1])) * STEP[name]
        # keep the depth of Gaussians with a close neighbour in depth
        tied = ids[~depth_free[ids]]
        v["means"][tied] -= np.outer(v["means"][tied] @ axis, axis)
        sides = []
        for s in (1.0, -1.0):
            scp = sc.subset(np.arange(n))
            for k, name in enumerate(("means", "log_scales", "quats", "opacity_logits", "sh")):
                arr = getattr(scp, name)
                d = v[list(GROUPS)[k]].reshape(arr.shape)
                setattr(scp, name, (arr.astype(np.float64) + s * d).astype(np.float32))
            sides.append(scp)
        # the discrete path must not change between the two sides
        same = True
        for scp in sides:
            kq = O.keypath(cam, scp)
            same &= all(np.array_equal(kq[key], kp[key]) for key in ("rect", "touched", "radius"))
        if not same:
            continue
        lp = _loss(_leaves(sides[0], dtype), cam, dtype, dimg_t)
        lm = _loss(_leaves(sides[1], dtype), cam, dtype, dimg_t)
        fd = (lp - lm) / 2.0
        # the perturbation actually applied: the FP32 values' difference
        ad = 0.0
        for k, name in enumerate(GROUPS):
            attr = ("means", "log_scales", "quats", "opacity_logits", "sh")[k]
            step = (getattr(sides[0], attr).astype(np.float64) - getattr(sides[1], attr).astype(np.float64)) / 2
            ad += float((g[name] * step.reshape(n, -1)).sum())
        print(f"direction {done}: autograd {ad:+.6e}, central difference {fd:+.6e}")
        assert abs(fd - ad) <= FD_RTOL * abs(ad) + FD_ATOL, (fd, ad)
        done += 1
    assert done == N_DIR, f"only {done} of {tries} directions kept the discrete path"

"""One clone-and-prune step (adaptive density control, Sec. II-A) through the
C ABI against the oracle, bit for bit: the kept Gaussians, the clones in
gradient order, the padding, the zeroed moments and the 16-bit SH shadow.
The screen-space gradient statistic is checked against the oracle's sum of
norms, and a trainer keeps training after it changed its Gaussian count."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S

pytestmark = pytest.mark.gpu

THR = float(np.float32(math.log(0.005 / 0.995)))


def _inputs(n, seed, kept_frac, tie_levels=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = rng.normal(0, 1, 59 * n).astype(np.float32)
    logit = np.where(rng.random(n) < kept_frac, rng.uniform(THR, 4, n), rng.uniform(-12, THR, n))
    logit[rng.random(n) < 0.01] = THR                          # exactly at the threshold: kept
    flat[10 * n:11 * n] = logit.astype(np.float32)
    m = rng.normal(0, 1e-3, 59 * n).astype(np.float32)
    v = rng.random(59 * n).astype(np.float32) * 1e-6
    g = rng.exponential(1e-4, n).astype(np.float32)
    if tie_levels:
        g = (np.floor(g / 1e-4 * tie_levels) / tie_levels).astype(np.float32)   # many equal values
    g[rng.random(n) < 0.02] = -1.0
    g[rng.random(n) < 0.02] = np.nan
    return flat, m, v, g


def _run(n, flat, m, v, g, thr, n_clone, capacity=None, shadow=None):
    dev = "cuda"
    cap = n + n_clone + 3 if capacity is None else capacity
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    p2 = torch.full((59 * max(cap, 1),), 7.0, device=dev)
    m2 = torch.full_like(p2, 7.0)
    v2 = torch.full_like(p2, 7.0)
    sh2 = None
    if shadow is not None:
        sh2 = torch.zeros(48 * max(cap, 1), dtype=torch.bfloat16 if shadow == L.GS_BF16 else torch.float16,
                          device=dev)
    ws = torch.empty(L.gs_densify_workspace(n) // 4 + 64, dtype=torch.float32, device=dev)
    n_out = torch.full((1,), -1, dtype=torch.int32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    L.gs_densify(n, t(flat), t(m), t(v), t(g), thr, n_clone, cap, p2, m2, v2, sh2,
                 shadow if shadow is not None else L.GS_BF16, n_out, ws, err)
    torch.cuda.synchronize()
    n2 = int(n_out.item())
    out = [x[:59 * n2].cpu().numpy() for x in (p2, m2, v2)]
    return n2, out, (sh2[:48 * n2].cpu() if sh2 is not None else None), int(err.item())


CASES = {
    # name: (N, seed, kept fraction, clones, tie levels)
    "2pct-4000": (4000, 1, 0.9, 80, None),
    "ties-4000": (4000, 2, 0.7, 80, 4),
    "ragged-300001": (300001, 3, 0.95, 6000, 16),
    "more-clones-than-kept": (64, 4, 0.3, 100, None),
    "no-clones": (1001, 5, 0.5, 0, None),
}


@pytest.mark.parametrize("case", list(CASES))
def test_densify_matches_oracle(case):
    n, seed, kf, n_clone, ties = CASES[case]
    flat, m, v, g = _inputs(n, seed, kf, ties)
    p_ref, m_ref, v_ref, n_ref = O.densify_prune(flat, m, v, g, n, THR, n_clone)
    n2, (p2, m2, v2), _, err = _run(n, flat, m, v, g, THR, n_clone)
    assert err == 0
    assert n2 == n_ref and n2 % 4 == 0
    assert np.array_equal(p2, p_ref)
    assert np.array_equal(m2, m_ref)
    assert np.array_equal(v2, v_ref)


@pytest.mark.parametrize("shadow", [L.GS_BF16, L.GS_F16])
def test_densify_writes_the_rounded_shadow(shadow):
    n = 2001
    flat, m, v, g = _inputs(n, 6, 0.8)
    p_ref, _, _, n_ref = O.densify_prune(flat, m, v, g, n, THR, 40)
    n2, (p2, _, _), sh2, err = _run(n, flat, m, v, g, THR, 40, shadow=shadow)
    assert err == 0 and n2 == n_ref
    dt = torch.bfloat16 if shadow == L.GS_BF16 else torch.float16
    want = torch.from_numpy(p_ref[11 * n2:]).to(dt)            # round to nearest even on the CPU
    assert torch.equal(sh2.view(torch.int16), want.view(torch.int16))


def test_padding_and_all_pruned():
    # 5 kept, 2 clones: 7 -> padded to 8 with an invisible copy of the first kept
    n = 12
    flat, m, v, g = _inputs(n, 7, 0.0)
    logit = flat[10 * n:11 * n]
    logit[[1, 3, 4, 8, 11]] = 0.5
    p_ref, m_ref, v_ref, n_ref = O.densify_prune(flat, m, v, g, n, THR, 2)
    n2, (p2, m2, v2), _, err = _run(n, flat, m, v, g, THR, 2)
    assert err == 0 and n2 == n_ref == 8
    assert p2[10 * 8 + 7] == np.float32(-30.0)
    assert np.array_equal(p2, p_ref) and np.array_equal(m2, m_ref) and np.array_equal(v2, v_ref)
    # nothing kept: count 0
    logit[:] = -20.0
    n2, _, _, err = _run(n, flat, m, v, g, THR, 2)
    assert err == 0 and n2 == 0
    # no Gaussians at all
    n2, _, _, err = _run(0, np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                         np.zeros(0, np.float32), THR, 0)
    assert err == 0 and n2 == 0


def test_capacity_too_small_is_reported():
    n = 400
    flat, m, v, g = _inputs(n, 8, 1.0)
    n2, _, _, err = _run(n, flat, m, v, g, THR, 40, capacity=n)
    assert err & L.GS_EW_CAPACITY and n2 == 0


def test_screen_grad_norm_accumulates_over_views_and_calls():
    V, n = 3, 1001
    rng = np.random.Generator(np.random.PCG64(9))
    g2 = rng.normal(0, 1e-3, V * n * 12).astype(np.float32)
    ref = O.screen_grad_norm(g2, V, n)
    out = torch.zeros(n, device="cuda")
    g2d = torch.from_numpy(g2).cuda()
    L.gs_grad2d_norm(V, n, g2d, out)
    L.gs_grad2d_norm(V, n, g2d, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.allclose(got, 2 * ref, rtol=1e-5, atol=0)


def test_trainer_densifies_and_keeps_training():
    """Two tracked steps, one clone-and-prune (2% clones, opacity < 0.005
    dropped), two more steps: the new state is the oracle's, bit for bit,
    and the steps after it run clean."""
    scene = S.uniform_scene(2000, 3)
    cams = [S.front_camera(112, 72)]
    tgt = torch.from_numpy(S.random_image(112, 72, seed=20).ravel()).cuda()
    params = P.to_device_params(scene)
    n = scene.n
    lo = params[10 * n:10 * n + n // 10]
    lo.fill_(-8.0)                                             # a tenth of the Gaussians nearly transparent
    tr = P.Trainer(cams, params, n, tgt, rgb_dtype=L.GS_BF16, sh_storage=L.GS_BF16,
                   schedule=P.Schedule("count"))
    tr.track_screen_grad()
    for _ in range(2):
        tr.step()
    torch.cuda.synchronize()
    assert tr.frame.check_errors() == 0
    p, m, v, g = (x.cpu().numpy() for x in (tr.p, tr.m, tr.v, tr.grad_norm[:n]))
    assert (g > 0).sum() > n // 4
    p_ref, m_ref, v_ref, n_ref = O.densify_prune(p, m, v, g, n, THR, int(0.02 * n))
    n2 = tr.densify(0.02, 0.005)
    assert n2 == n_ref == tr.N and n2 < n
    assert np.array_equal(tr.p.cpu().numpy(), p_ref)
    assert np.array_equal(tr.m.cpu().numpy(), m_ref)
    assert np.array_equal(tr.v.cpu().numpy(), v_ref)
    assert torch.equal(tr.sh_shadow.cpu().view(torch.int16),
                       torch.from_numpy(p_ref[11 * n2:]).to(torch.bfloat16).view(torch.int16))
    for _ in range(2):
        loss = tr.step()
    torch.cuda.synchronize()
    assert tr.frame.check_errors() == 0
    assert math.isfinite(float(loss.item()))
    assert torch.isfinite(tr.p).all()
    assert float(tr.grad_norm[:n2].sum()) > 0                  # the statistic restarted and accumulates again

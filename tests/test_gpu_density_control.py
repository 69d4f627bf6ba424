"""Workload-sensitive density control (Sec. III-C) through the C ABI against
the oracle.  Densities, nearest neighbours and their distances, the k-nearest
mean distance, the low/high thresholds and the spawned points are exact (FP32
with every operation rounded; integer sums); merged positions and scales go
through exp/log, so they are compared within 1e-6; d_merge is an FP64 sum in
no fixed order, compared within 1e-12 relative, and the test checks that no
candidate pair lies so close to it that the decision could flip."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import scenes as S

pytestmark = pytest.mark.gpu

ALPHA, BETA, GAMMA, ALPHA_D = 1.0, 1.0, 1.0, 1.5


def _stats(P, r, k):
    n = len(P)
    dev = "cuda"
    rho = torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev)
    nn = torch.full_like(rho, -7)
    dbar = torch.full((max(n, 1),), -1.0, device=dev)
    dnn = torch.full_like(dbar, -1.0)
    thr = torch.zeros(3, dtype=torch.float64, device=dev)
    ws = torch.empty(L.gs_density_workspace(n) // 4 + 64, dtype=torch.float32, device=dev)
    L.gs_density_stats(n, torch.from_numpy(np.ascontiguousarray(P, np.float32)).to(dev).view(-1), r, k,
                       rho, dbar, nn, dnn, (ALPHA, BETA, GAMMA), thr, ws)
    torch.cuda.synchronize()
    return (rho[:n].cpu().numpy(), dbar[:n].cpu().numpy(), nn[:n].cpu().numpy(), dnn[:n].cpu().numpy(),
            thr.cpu().numpy())


def _dup(n, seed):
    P = S.uniform_scene(n, seed).means
    return np.repeat(P, 3, axis=0)[: n]


STATS_CASES = {
    "skewed-20000": (lambda: S.skewed_scene(20_000, 0).means, 0.02, 3),
    "uniform-5000-k5": (lambda: S.uniform_scene(5_000, 1).means, 0.1, 5),
    "duplicates-3000-k8": (lambda: _dup(3000, 2), 0.08, 8),
    "ragged-1001": (lambda: S.skewed_scene(1001, 4).means, 0.05, 3),
    "two-points": (lambda: S.uniform_scene(2, 3).means, 0.1, 3),
    "one-point": (lambda: S.uniform_scene(1, 3).means, 0.1, 3),
}


@pytest.mark.parametrize("name", list(STATS_CASES))
def test_density_stats_match_oracle(name):
    make, r, k = STATS_CASES[name]
    P = np.ascontiguousarray(make(), np.float32)
    rho, dbar, nn, dnn, thr = _stats(P, r, k)
    rho_o, dbar_o, nn_o, dnn_o = O.density_stats(P, r, k)
    assert np.array_equal(rho, rho_o)
    assert np.array_equal(nn, nn_o)
    assert np.array_equal(dnn, dnn_o)
    assert np.array_equal(dbar, dbar_o)
    lo, hi, dm = O.density_thresholds(rho_o, dnn_o, ALPHA, BETA, GAMMA)
    assert thr[0] == lo and thr[1] == hi                       # exact: integer sums
    assert abs(thr[2] - dm) <= 1e-12 * max(abs(dm), 1e-30)


def test_density_stats_at_full_size_on_sampled_points():
    """3M skewed Gaussians (the benchmark scene): 48 sampled points against
    all 3M by brute force; thresholds from the device's own densities."""
    P = np.ascontiguousarray(S.skewed_scene(3_000_000, 0).means, np.float32)
    r, k = 0.005, 3
    rho, dbar, nn, dnn, thr = _stats(P, r, k)
    rng = np.random.default_rng(5)
    for i in rng.choice(len(P), 48, replace=False):
        assert (rho[i], dbar[i], nn[i], dnn[i]) == O.density_point(P, i, r, k)
    lo, hi, dm = O.density_thresholds(rho.astype(np.int64), dnn, ALPHA, BETA, GAMMA)
    assert thr[0] == lo and thr[1] == hi
    assert abs(thr[2] - dm) <= 1e-12 * dm


def _inputs(P, seed):
    n = len(P)
    rng = np.random.default_rng(seed)
    flat = rng.normal(0, 1, 59 * n).astype(np.float32)
    flat[:3 * n] = np.asarray(P, np.float32).ravel()
    flat[3 * n:6 * n] = rng.normal(-4, 0.5, 3 * n).astype(np.float32)
    m = rng.normal(0, 1e-3, 59 * n).astype(np.float32)
    v = rng.random(59 * n).astype(np.float32) * 1e-6
    z, u = S.density_draws(n, seed)
    return flat, m, v, z, u


def _control(n, flat, m, v, z, u, r, k, delta, capacity=None, shadow=None):
    dev = "cuda"
    cap = 2 * n + 3 if capacity is None else capacity
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    p2 = torch.full((59 * max(cap, 1),), 7.0, device=dev)
    m2, v2 = torch.full_like(p2, 7.0), torch.full_like(p2, 7.0)
    sh = None
    if shadow is not None:
        sh = torch.zeros(48 * max(cap, 1), dtype=torch.bfloat16, device=dev)
    n_out = torch.full((1,), -1, dtype=torch.int32, device=dev)
    thr = torch.zeros(3, dtype=torch.float64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(L.gs_density_workspace(n) // 4 + 64, dtype=torch.float32, device=dev)
    L.gs_density_control(n, t(flat), t(m), t(v), t(z.ravel()), t(u.ravel()), r, k, ALPHA, BETA, ALPHA_D, delta,
                         GAMMA, cap, p2, m2, v2, sh, L.GS_BF16, n_out, thr, ws, err)
    torch.cuda.synchronize()
    n2 = int(n_out.item())
    return (n2, [x[:59 * n2].cpu().numpy() for x in (p2, m2, v2)], sh[:48 * n2].cpu() if sh is not None else None,
            thr.cpu().numpy(), int(err.item()))


def _split(a, n):
    return np.split(a, np.cumsum([3 * n, 3 * n, 4 * n, n]))


CONTROL_CASES = {
    "skewed-20000": (lambda: S.skewed_scene(20_000, 1).means, 0.02),
    "skewed-4001": (lambda: S.skewed_scene(4001, 2).means, 0.02),
    "uniform-3000": (lambda: S.uniform_scene(3000, 3).means, 0.25),
}


@pytest.mark.parametrize("case", list(CONTROL_CASES))
def test_density_control_matches_oracle(case):
    make, r = CONTROL_CASES[case]
    P = make()
    n = len(P)
    k, delta = 3, 0.004
    flat, m, v, z, u = _inputs(P, 9)
    p_ref, m_ref, v_ref, n_ref, info = O.density_control(flat, m, v, n, r, k, ALPHA, BETA, ALPHA_D, delta,
                                                          GAMMA, z, u)
    # no mutual high-density pair within rounding of d_merge (the decision is robust)
    cand = info["high"] & info["high"][np.maximum(info["nn"], 0)]
    assert not np.any(cand & (np.abs(info["dnn"].astype(np.float64) - info["d_merge"]) <= 1e-9 * info["d_merge"]))
    assert info["n_merged"] > 0 and info["n_new"] > 0
    n2, (p2, m2, v2), sh, thr, err = _control(n, flat, m, v, z, u, r, k, delta, shadow=True)
    assert err == 0 and n2 == n_ref and n2 % 4 == 0
    assert thr[0] == info["rho_low"] and thr[1] == info["rho_high"]
    a, b = info["n_keep"], info["n_merged"]
    G, Gr = _split(p2, n2), _split(p_ref, n2)
    for g, w in enumerate((3, 3, 4, 1, 48)):
        x, y = G[g].reshape(n2, w), Gr[g].reshape(n2, w)
        assert np.array_equal(x[:a], y[:a]), g                       # untouched
        assert np.array_equal(x[a + b:], y[a + b:]), g               # spawned and padding: exact FP32
        if g in (0, 1):
            assert np.allclose(x[a:a + b], y[a:a + b], rtol=0, atol=1e-6), g   # exp / log
        else:
            assert np.array_equal(x[a:a + b], y[a:a + b]), g
    assert np.array_equal(m2, m_ref) and np.array_equal(v2, v_ref)
    want = torch.from_numpy(p2[11 * n2:]).to(torch.bfloat16)
    assert torch.equal(sh.view(torch.int16), want.view(torch.int16))


def test_density_control_capacity_and_empty():
    P = S.skewed_scene(2000, 5).means
    flat, m, v, z, u = _inputs(P, 3)
    n2, _, _, _, err = _control(2000, flat, m, v, z, u, 0.02, 3, 0.004, capacity=100)
    assert err & L.GS_EW_CAPACITY and n2 == 0
    e = np.zeros(0, np.float32)
    n2, _, _, thr, err = _control(0, e, e, e, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                                  0.02, 3, 0.004)
    assert n2 == 0 and err == 0


def test_bad_arguments_are_refused():
    P = np.zeros((8, 3), np.float32)
    for r, k in ((0.0, 3), (0.1, 0), (0.1, 9)):
        with pytest.raises(L.GsError):
            _stats(P, r, k)

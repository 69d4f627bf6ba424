"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  Each one checks the oracle against something
other than itself: closed forms of special cases (Sec. II-A's G(x), Sigma' and
blending equations), invariants of front-to-back blending, textbook tables,
scipy's spherical harmonics, brute-force enumeration written independently in
numpy, and central finite differences of the oracle's own forward.
"""
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_14564_gb300 import scenes as S

GOLDEN = Path(__file__).resolve().parent / "golden"
Y00 = 0.5 / math.sqrt(math.pi)


def one_scene(means, log_scales, quats, logits, sh):
    n = len(means)
    f = lambda a, s: np.ascontiguousarray(np.asarray(a, np.float64).reshape(s), np.float32)
    return S.Scene(f(means, (n, 3)), f(log_scales, (n, 3)), f(quats, (n, 4)),
                   f(logits, (n,)), f(sh, (n, 16, 3)))


def dc_sh(rgb):
    """SH block whose DC term gives colour `rgb` (0.5 + Y00 k = rgb)."""
    sh = np.zeros((16, 3))
    sh[0] = (np.asarray(rgb, np.float64) - 0.5) / Y00
    return sh


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def f32(x):
    """The float32 value a scene stores for x."""
    return float(np.float32(x))


def s32(s):
    """The scale a float32-stored log-scale of log(s) decodes to."""
    return math.exp(f32(math.log(s)))


# ---------------------------------------------------------------------------
# Single isotropic Gaussian on the optical axis: closed form
# ---------------------------------------------------------------------------

def test_single_isotropic_gaussian_closed_form():
    cam = S.front_camera(64, 64)
    s, logit, rgb = 0.05, 0.5, (0.7, 0.3, 0.55)
    sc = one_scene([[0, 0, 0]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [logit], [dc_sh(rgb)])
    r = O.forward(cam, sc)
    kp = r["kp"]
    z = 3.0
    f = float(np.float32(cam.fx))
    var = (f * s32(s) / z) ** 2 + 0.3
    rad = math.ceil(3 * math.sqrt(var))
    assert kp["radius"][0] == rad == 4
    # rect: floor((u - r)/16), floor((u + r + 15)/16) with u = 32
    assert list(kp["rect"][0]) == [1, 1, 3, 3] and kp["touched"][0] == 4
    o = sigmoid(f32(logit))
    rgb_exp = 0.5 + Y00 * sc.sh[0, 0].astype(np.float64)      # float32-stored DC term
    ys, xs = np.mgrid[0:64, 0:64]
    rho2 = (xs + 0.5 - 32.0) ** 2 + (ys + 0.5 - 32.0) ** 2
    alpha = np.minimum(0.99, o * np.exp(-0.5 * rho2 / var))
    inside = (xs >= 16) & (xs < 48) & (ys >= 16) & (ys < 48)      # the two-by-two tile block
    keep = inside & (alpha >= 1 / 255)
    expect = np.where(keep[None], alpha[None] * rgb_exp[:, None, None], 0.0)
    assert np.allclose(r["img"], expect, rtol=0, atol=1e-12)
    assert np.allclose(r["T_final"], np.where(keep, 1 - alpha, 1.0), atol=1e-12)
    assert np.array_equal(r["n_proc"], keep.astype(np.int32))
    assert r["flag"].sum() == 0


def test_single_gaussian_alpha_clamp():
    cam = S.front_camera(64, 64)
    s, logit = 0.5, 6.0
    sc = one_scene([[0, 0, 0]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [logit], [dc_sh((1, 1, 1))])
    r = O.forward(cam, sc, window=(30, 30, 34, 34))
    var = (float(np.float32(cam.fx)) * s32(s) / 3.0) ** 2 + 0.3
    a0 = sigmoid(f32(logit)) * math.exp(-0.5 * 0.5 / var)     # pixel (31, 31): rho^2 = 0.5
    assert a0 > 0.99
    c0 = 0.5 + Y00 * float(sc.sh[0, 0, 0])
    assert r["img"][0, 31, 31] == pytest.approx(0.99 * c0, abs=1e-12)
    assert r["T_final"][31, 31] == pytest.approx(0.01, abs=1e-12)


def test_single_gaussian_skip_threshold():
    """A Gaussian whose alpha is below 1/255 at a pixel leaves it untouched."""
    cam = S.front_camera(64, 64)
    s, logit = 0.05, -4.0         # o = 0.018
    sc = one_scene([[0, 0, 0]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [logit], [dc_sh((1, 1, 1))])
    r = O.forward(cam, sc)
    o = sigmoid(f32(logit))
    var = (float(np.float32(cam.fx)) * s32(s) / 3.0) ** 2 + 0.3
    ys, xs = np.mgrid[0:64, 0:64]
    a = o * np.exp(-0.5 * ((xs + 0.5 - 32) ** 2 + (ys + 0.5 - 32) ** 2) / var)
    inside = (xs >= 16) & (xs < 48) & (ys >= 16) & (ys < 48)
    touched = inside & (a >= 1 / 255)
    assert touched.sum() > 0 and (inside & ~touched).sum() > 0
    assert np.all(r["img"][0][~touched] == 0.0)
    c0 = 0.5 + Y00 * float(sc.sh[0, 0, 0])
    assert np.allclose(r["img"][0][touched], c0 * a[touched], atol=1e-12)


# ---------------------------------------------------------------------------
# Two Gaussians: blending order follows depth
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("swap", [False, True])
def test_two_gaussians_order(swap):
    cam = S.front_camera(64, 64)
    z1, z2 = (0.0, 0.5) if not swap else (0.5, 0.0)
    s, l1, l2 = 0.08, 0.3, 1.2
    c1, c2 = (0.9, 0.2, 0.1), (0.1, 0.3, 0.8)
    sc = one_scene([[0, 0, z1], [0, 0, z2]], [[math.log(s)] * 3] * 2, [[1, 0, 0, 0]] * 2,
                   [l1, l2], [dc_sh(c1), dc_sh(c2)])
    r = O.forward(cam, sc, window=(31, 31, 32, 32))
    f = float(np.float32(cam.fx))

    def alpha(zw, logit):
        var = (f * s32(s) / (3.0 + f32(zw))) ** 2 + 0.3
        return sigmoid(f32(logit)) * math.exp(-0.5 * 0.5 / var)

    a1, a2 = alpha(z1, l1), alpha(z2, l2)
    col = 0.5 + Y00 * sc.sh[:, 0, :].astype(np.float64)        # float32-stored DC terms
    front, back = ((a1, col[0]), (a2, col[1])) if z1 < z2 else ((a2, col[1]), (a1, col[0]))
    expect = front[1] * front[0] + back[1] * back[0] * (1 - front[0])
    assert np.allclose(r["img"][:, 31, 31], expect, atol=1e-12)
    assert r["T_final"][31, 31] == pytest.approx((1 - a1) * (1 - a2), abs=1e-12)
    assert r["n_proc"][31, 31] == 2


# ---------------------------------------------------------------------------
# Transmittance identity: with unit colours, img = (1 - T_final) + T_final bg
# ---------------------------------------------------------------------------

def test_transmittance_identity():
    sc = S.uniform_scene(3000, seed=11)
    sc.sh[:] = 0.0
    sc.sh[:, 0, :] = 0.5 / Y00
    cam = S.front_camera(96, 80)
    cam.bg = (0.25, 0.5, 0.75)
    r = O.forward(cam, sc)
    T = r["T_final"]
    col = r["proj"]["rgb"][r["kp"]["touched"] > 0][0]      # every Gaussian has this colour
    assert np.all(np.abs(col - 1.0) < 1e-6)
    for ch in range(3):
        assert np.allclose(r["img"][ch], col[ch] * (1 - T) + T * cam.bg[ch], atol=1e-12)
    assert (T < 0.5).mean() > 0.05          # the scene does cover pixels
    # the stop rule: nothing ends below 1e-4
    assert T.min() >= 1e-4


def test_transmittance_stop_rule():
    """Ten identical opaque Gaussians: stop before T would fall below 1e-4."""
    cam = S.front_camera(64, 64)
    n = 10
    sc = one_scene([[0, 0, 0.01 * k] for k in range(n)], [[math.log(0.5)] * 3] * n,
                   [[1, 0, 0, 0]] * n, [1.5] * n, [dc_sh((1, 1, 1))] * n)
    r = O.forward(cam, sc, window=(31, 31, 32, 32))
    f = float(np.float32(cam.fx))
    T, k_last = 1.0, 0
    for k in range(n):
        var = (f * s32(0.5) / (3.0 + f32(0.01 * k))) ** 2 + 0.3
        a = min(0.99, sigmoid(f32(1.5)) * math.exp(-0.5 * 0.5 / var))
        if T * (1 - a) < 1e-4:
            break
        T *= 1 - a
        k_last = k + 1
    assert k_last < n                     # the rule fired
    assert r["n_proc"][31, 31] == k_last
    assert r["T_final"][31, 31] == pytest.approx(T, rel=1e-12)


# ---------------------------------------------------------------------------
# Sigma' = J W Sigma W^T J^T (+0.3 I): special cases
# ---------------------------------------------------------------------------

def test_cov2d_axis_aligned_and_rotated():
    cam = S.front_camera(64, 64)
    f = float(np.float32(cam.fx))
    sx, sy, sz = 0.05, 0.02, 0.07
    th = 0.6
    sc = one_scene([[0, 0, 0], [0, 0, 0]], [[math.log(sx), math.log(sy), math.log(sz)]] * 2,
                   [[1, 0, 0, 0], [math.cos(th / 2), 0, 0, math.sin(th / 2)]], [0, 0],
                   [np.zeros((16, 3))] * 2)
    kp = O.keypath(cam, sc)
    pr = O.project(cam, sc, kp)
    D = np.diag([(f * s32(sx) / 3) ** 2, (f * s32(sy) / 3) ** 2])
    for i, ang in enumerate([0.0, 2 * math.atan2(float(sc.quats[1, 3]), float(sc.quats[1, 0]))]):
        Rz = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
        S2 = Rz @ D @ Rz.T + 0.3 * np.eye(2)
        K = np.linalg.inv(S2)
        A, B, C = pr["conic"][i]
        assert np.allclose([A, B, C], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-12)
        # FP32 key path agrees with FP64 to float precision
        assert np.allclose(kp["cov2d"][i], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=2e-6, atol=1e-6)


def test_cov2d_off_axis_jacobian():
    """Off-axis isotropic Gaussian: Sigma' = s^2 J J^T + 0.3 I with the third
    column of J = -f x / z^2 (pins the projective Jacobian)."""
    cam = S.front_camera(64, 64)
    f = float(np.float32(cam.fx))
    s, x, y = 0.03, 0.7, -0.4
    sc = one_scene([[x, y, 0.0]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [0], [np.zeros((16, 3))])
    kp = O.keypath(cam, sc)
    pr = O.project(cam, sc, kp)
    z = 3.0
    x, y = f32(x), f32(y)
    J = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
    S2 = s32(s) ** 2 * J @ J.T + 0.3 * np.eye(2)
    K = np.linalg.inv(S2)
    assert np.allclose(pr["conic"][0], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-12)
    assert np.allclose(pr["mean2d"][0], [f * x / z + 32, f * y / z + 32], rtol=1e-12)


def test_keypath_culling_and_status():
    cam = S.front_camera(64, 64)
    sc = one_scene([[0, 0, -2.9], [0, 0, -4.0], [50, 0, 0], [0, 0, 0], [0, float("nan"), 0]],
                   [[-3] * 3] * 5, [[1, 0, 0, 0]] * 5, [0] * 5, [np.zeros((16, 3))] * 5)
    kp = O.keypath(cam, sc)
    # z = 0.1 (< znear), z = -1 (behind), far off-screen, visible, NaN
    assert list(kp["touched"] > 0) == [False, False, False, True, False]
    assert list(kp["status"]) == [0, 0, 0, 0, 1]


def test_exp_spec_accuracy():
    xs = np.linspace(-20, 20, 4001, dtype=np.float32)
    got = np.array([O.exp_spec(float(x)) for x in xs], np.float64)
    ref = np.exp(xs.astype(np.float64))
    assert np.max(np.abs(got - ref) / ref) < 4 * 2.0 ** -23


# ---------------------------------------------------------------------------
# Spherical harmonics
# ---------------------------------------------------------------------------

def _sphere_quadrature(nz=24, nphi=48):
    zs, wz = np.polynomial.legendre.leggauss(nz)
    phis = 2 * np.pi * np.arange(nphi) / nphi
    pts, w = [], []
    for z, wzz in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            pts.append((r * math.cos(ph), r * math.sin(ph), z))
            w.append(wzz * 2 * np.pi / nphi)
    return np.array(pts), np.array(w)


def test_sh_orthonormal_by_quadrature():
    pts, w = _sphere_quadrature()
    Y = np.array([O.sh_basis(*p)[0] for p in pts])
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_textbook_table():
    rows = [l.split(None, 3) for l in (GOLDEN / "real_sh_degree3.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    rng = np.random.default_rng(5)
    for _ in range(20):
        v = rng.normal(size=3)
        x, y, z = v / np.linalg.norm(v)
        Y, _ = O.sh_basis(x, y, z)
        for idx, l, m, expr in rows:
            val = eval(expr, {"sqrt": math.sqrt, "pi": math.pi, "x": x, "y": y, "z": z})
            assert Y[int(idx)] == pytest.approx(val, abs=1e-13), (l, m)


def test_sh_matches_scipy_complex_harmonics():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(6)
    for _ in range(10):
        v = rng.normal(size=3)
        x, y, z = v / np.linalg.norm(v)
        theta, phi = math.acos(z), math.atan2(y, x)
        Y, _ = O.sh_basis(x, y, z)
        for l in range(4):
            for m in range(-l, l + 1):
                c = sp.sph_harm_y(l, abs(m), theta, phi)
                if m == 0:
                    ref = c.real
                elif m > 0:
                    ref = math.sqrt(2) * (-1) ** m * c.real
                else:
                    ref = math.sqrt(2) * (-1) ** m * c.imag
                assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-12)


def test_sh_gradient_central_differences():
    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(5):
        p = rng.normal(size=3)
        _, G = O.sh_basis(*p)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            fd = (O.sh_basis(*(p + e))[0] - O.sh_basis(*(p - e))[0]) / (2 * h)
            assert np.allclose(G[:, k], fd, atol=1e-7)


# ---------------------------------------------------------------------------
# Tile lists: brute force in numpy
# ---------------------------------------------------------------------------

def test_tile_lists_brute_force():
    sc = S.uniform_scene(400, seed=3)
    sc.log_scales += 1.0
    cam = S.front_camera(72, 40)    # ragged: 5 x 3 tiles, partial last column and row
    kp = O.keypath(cam, sc)
    TX = cam.tiles_x
    trip = []
    for i in range(sc.n):
        if kp["touched"][i] <= 0:
            continue
        x0, y0, x1, y1 = kp["rect"][i]
        assert (x1 - x0) * (y1 - y0) == kp["touched"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                trip.append((ty * TX + tx, int(kp["depth"][i:i + 1].view(np.uint32)[0]), i))
    trip = np.array(trip, dtype=np.int64)
    order = np.lexsort((trip[:, 2], trip[:, 1], trip[:, 0]))
    trip = trip[order]
    counts = O.tile_counts(cam, kp)
    assert counts.sum() == len(trip) == kp["touched"].sum()
    start = 0
    for t in range(cam.n_tiles):
        ids = O.tile_list(kp, t % TX, t // TX)
        assert len(ids) == counts[t]
        assert np.array_equal(ids, trip[start:start + counts[t], 2])
        start += counts[t]


def test_tile_list_depth_ties_by_index():
    cam = S.front_camera(32, 32)
    sc = one_scene([[0, 0, 0]] * 3, [[-3] * 3] * 3, [[1, 0, 0, 0]] * 3, [0] * 3,
                   [np.zeros((16, 3))] * 3)
    kp = O.keypath(cam, sc)
    assert np.array_equal(O.tile_list(kp, 0, 0), [0, 1, 2])


# ---------------------------------------------------------------------------
# Gradients: central differences of the FP64 forward
# ---------------------------------------------------------------------------

def _grad_scene(seed):
    rng = np.random.default_rng(seed)
    n = 12
    means = np.c_[rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(-0.3, 0.3, n)]
    ls = rng.normal(-1.6, 0.25, (n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(-0.5, 0.6, n)
    sh = rng.normal(0, 0.2, (n, 16, 3))
    sh[0, 0, 1] = -4.0            # a colour clamped at 0 (zero SH gradient)
    logits[1] = 7.0               # an opacity clamped at 0.99 near its centre
    return one_scene(means, ls, q, logits, sh)


def _loss(cam, sc, kp, p64, dimg):
    pr = O.project(cam, sc, kp, p64)
    r = O.render(cam, kp, pr)
    return float(np.sum(r["img"] * dimg)), r


@pytest.fixture(scope="module")
def grad_case():
    cam = S.front_camera(32, 32)
    for seed in range(50):
        sc = _grad_scene(seed)
        kp = O.keypath(cam, sc)
        pr = O.project(cam, sc, kp)
        r = O.render(cam, kp, pr, margin_alpha=1e-3, margin_T=1e-2)
        ok = (r["flag"].sum() == 0 and (kp["touched"] > 0).all()
              and np.all(np.abs(pr["rgb_pre"]) > 1e-3))
        if ok:
            dimg = S.random_cotangent((3, 32, 32), seed=seed)
            return cam, sc, kp, pr, dimg
    pytest.fail("no threshold-free gradient scene found")


def test_render_bwd_central_differences(grad_case):
    cam, sc, kp, pr, dimg = grad_case
    g = O.render_bwd(cam, kp, pr, dimg)
    h = 1e-6
    fields = [("mean2d", 0), ("mean2d", 1), ("conic", 0), ("conic", 1), ("conic", 2),
              ("opac", None), ("rgb", 0), ("rgb", 1), ("rgb", 2)]
    for i in range(sc.n):
        for q, (name, col) in enumerate(fields):
            vals = []
            for sgn in (+1, -1):
                p2 = {k: v.copy() for k, v in pr.items()}
                if col is None:
                    p2[name][i] += sgn * h
                else:
                    p2[name][i, col] += sgn * h
                vals.append(float(np.sum(O.render(cam, kp, p2)["img"] * dimg)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[i, q] == pytest.approx(fd, rel=1e-5, abs=1e-8), (i, name, col)


def test_full_gradient_central_differences(grad_case):
    cam, sc, kp, pr, dimg = grad_case
    g2 = O.render_bwd(cam, kp, pr, dimg)
    g = O.project_bwd(cam, sc, kp, g2)
    base = {"means": sc.means.astype(np.float64), "log_scales": sc.log_scales.astype(np.float64),
            "quats": sc.quats.astype(np.float64),
            "opacity_logits": sc.opacity_logits.astype(np.float64),
            "sh": sc.sh.astype(np.float64).reshape(sc.n, 48)}
    h = 1e-6
    off = 0
    for name, w in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)):
        for i in range(sc.n):
            for k in range(w):
                vals = []
                for sgn in (+1, -1):
                    p = {kk: vv.copy() for kk, vv in base.items()}
                    if w == 1:
                        p[name][i] += sgn * h
                    else:
                        p[name][i, k] += sgn * h
                    vals.append(_loss(cam, sc, kp, p, dimg)[0])
                fd = (vals[0] - vals[1]) / (2 * h)
                got = g[off + i * w + k]
                assert got == pytest.approx(fd, rel=1e-5, abs=1e-8), (name, i, k)
        off += w * sc.n
    # the clamped colour channel has no SH gradient; the clamped opacity
    # Gaussian still has colour gradients
    dsh = g[11 * sc.n:].reshape(sc.n, 16, 3)
    assert np.all(dsh[0, :, 1] == 0.0)


# ---------------------------------------------------------------------------
# L1, Adam, MLP, features
# ---------------------------------------------------------------------------

def test_l1_closed_form():
    img = np.array([0.5, 0.2, 0.9, 0.4])
    tgt = np.array([0.5, 0.3, 0.1, 0.4])
    loss, d = O.l1(img, tgt)
    assert loss == pytest.approx((0.1 + 0.8) / 4, abs=1e-15)
    assert list(d) == [0.0, -0.25, 0.25, 0.0]


def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(1)
    n = 64
    p0 = rng.normal(size=n)
    g = rng.normal(size=n)
    g[0] = 0.0
    lr = np.full(n, 1e-3)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        p, m, v = O.adam(p, g, m, v, lr, step=t)
        # bias-corrected moments of a constant gradient are g and g^2 exactly
        expect = p0 - t * lr * g / (np.abs(g) + 1e-15)
        assert np.allclose(p, expect, rtol=0, atol=1e-13)


def test_adam_two_steps_closed_form():
    g1, g2 = np.array([0.3, -2.0]), np.array([-0.1, 4.0])
    lr = np.array([0.01, 0.02])
    p, m, v = O.adam(np.zeros(2), g1, np.zeros(2), np.zeros(2), lr, step=1)
    p, m, v = O.adam(p, g2, m, v, lr, step=2)
    m2 = 0.09 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step1 = lr * g1 / (np.abs(g1) + 1e-15)
    step2 = lr * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-15)
    assert np.allclose(p, -step1 - step2, rtol=1e-13)


def test_mlp_forward_hand_case():
    W1 = np.zeros((32, 8)); b1 = np.zeros(32); W2 = np.zeros(32)
    W1[0, 0] = 2.0; W1[1, 1] = -1.0; b1[1] = 0.5; W2[0] = 3.0; W2[1] = 4.0
    f = np.zeros((2, 8)); f[0, 0] = 1.5; f[0, 1] = 0.25; f[1, 1] = 2.0
    y = O.mlp_fwd(f, W1, b1, W2, 0.1)
    # row 0: relu(3) * 3 + relu(0.25) * 4 + 0.1; row 1: relu(-1.5) = 0 -> 0.1
    assert np.allclose(y, [9.0 + 1.0 + 0.1, 0.1], atol=1e-15)


def test_mlp_gradient_central_differences():
    rng = np.random.default_rng(2)
    n = 40
    f = rng.normal(size=(n, 8))
    tgt = rng.normal(size=n)
    W = rng.normal(0, 0.4, 321)
    unpack = lambda w: (w[:256].reshape(32, 8), w[256:288], w[288:320], w[320:321])
    loss, g = O.mlp_loss_grad(f, tgt, *unpack(W))
    h = 1e-6
    for k in range(321):
        e = np.zeros(321); e[k] = h
        fd = (O.mlp_loss_grad(f, tgt, *unpack(W + e))[0] - O.mlp_loss_grad(f, tgt, *unpack(W - e))[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    y = O.mlp_fwd(f, *unpack(W))
    assert loss == pytest.approx(np.mean((y - tgt) ** 2), rel=1e-13)


def test_tile_features_single_gaussian_and_edge():
    cam = S.front_camera(40, 40)         # 3 x 3 tiles, last row and column 8 px
    s, logit = 0.05, 0.4
    sc = one_scene([[0, 0, 0]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [logit], [np.zeros((16, 3))])
    kp = O.keypath(cam, sc)
    pr = O.project(cam, sc, kp)
    f = O.tile_features(cam, kp, pr, 1, 1)
    o = sigmoid(f32(logit))
    var = (float(np.float32(cam.fx)) * s32(s) / 3) ** 2 + 0.3
    cov = min(1.0, math.pi * var / 256)
    assert f[0] == pytest.approx(math.log(2))
    assert f[1] == pytest.approx(o) and f[2] == pytest.approx(o)
    assert f[3] == pytest.approx(cov, rel=1e-12)
    assert f[4] == pytest.approx(math.log1p(o * cov), rel=1e-12)
    assert f[5] == pytest.approx(math.log(2), rel=1e-12)       # sum of Th = Th_0 = 1
    assert f[6] == 1.0
    assert f[7] == pytest.approx(math.log1p(1600) / 16)
    fe = O.tile_features(cam, kp, pr, 2, 2)
    assert fe[6] == pytest.approx(64 / 256) and fe[0] == 0.0


def test_tile_features_saturation_sum():
    """f5 sums the expected transmittance while it stays at or above 1e-4."""
    cam = S.front_camera(32, 32)
    n = 30
    sc = one_scene([[0, 0, 0.001 * k] for k in range(n)], [[math.log(0.4)] * 3] * n,
                   [[1, 0, 0, 0]] * n, [3.0] * n, [np.zeros((16, 3))] * n)
    kp = O.keypath(cam, sc)
    pr = O.project(cam, sc, kp)
    f = O.tile_features(cam, kp, pr, 0, 0)
    Th, acc = 1.0, 0.0
    for k in range(n):
        if Th < 1e-4:
            break
        acc += Th
        dconic = pr["conic"][k, 0] * pr["conic"][k, 2] - pr["conic"][k, 1] ** 2
        cov = min(1.0, math.pi * math.sqrt(1 / dconic) / 256)
        Th *= 1 - min(0.99, pr["opac"][k] * cov)
    assert f[5] == pytest.approx(math.log1p(acc), rel=1e-12)


# --- densification (clone + prune) ------------------------------------------
def _dp_scene(n, seed):
    rng = np.random.default_rng(seed)
    flat = rng.normal(size=59 * n).astype(np.float32)
    m = rng.normal(size=59 * n).astype(np.float32)
    v = rng.random(59 * n).astype(np.float32)
    return flat, m, v


def test_densify_prune_by_hand():
    """Eight Gaussians, logits chosen around the threshold, gradients with a
    tie: the kept ones in index order, then the two largest gradients (the tie
    broken by index), moments zeroed for the clones only."""
    n = 8
    flat, m, v = _dp_scene(n, 0)
    thr = np.float32(-5.0)
    flat[10 * n:11 * n] = np.array([-6, -5, 0, 3, -5.0000005, 1, -7, 2], np.float32)
    g = np.array([0.9, 0.1, 0.5, 0.5, 9.0, np.nan, 0.2, 0.3], np.float32)
    f2, m2, v2, n2 = O.densify_prune(flat, m, v, g, n, thr, 2)
    keep = [1, 2, 3, 5, 7]                        # logit >= -5 (index 4 is just below)
    clones = [2, 3]                               # g: 0.5 (2), 0.5 (3): the tie by index; NaN is 0
    # 5 kept + 2 clones = 7; dropping 3 clones is impossible, so one pad: 8
    assert n2 == 8
    src = keep + clones + [keep[0]]
    for gi, (o, w) in enumerate(((0, 3), (3, 3), (6, 4), (10, 1), (11, 48))):
        got = f2[o * n2:(o + w) * n2].reshape(n2, w)
        ref = flat[o * n:(o + w) * n].reshape(n, w)[src]
        if gi == 3:
            ref = ref.copy()
            ref[7, 0] = -30.0
        assert np.array_equal(got, ref)
        mg = m2[o * n2:(o + w) * n2].reshape(n2, w)
        assert np.array_equal(mg[:5], m[o * n:(o + w) * n].reshape(n, w)[keep])
        assert not mg[5:].any()


def test_densify_prune_count_and_alignment():
    rng = np.random.default_rng(3)
    for n in (4, 100, 1000):
        flat, m, v = _dp_scene(n, n)
        g = rng.random(n).astype(np.float32)
        for k in (0, 1, 3, n // 50, n):
            f2, m2, v2, n2 = O.densify_prune(flat, m, v, g, n, np.float32(-1.0), k)
            kept = int((flat[10 * n:11 * n] >= -1.0).sum())
            assert n2 % 4 == 0 and kept <= n2 <= kept + min(k, kept) + 3
            assert f2.size == 59 * n2 and m2.size == 59 * n2 and v2.size == 59 * n2


def test_densify_prune_keeps_no_pruned_clone_and_handles_all_pruned():
    n = 12
    flat, m, v = _dp_scene(n, 5)
    flat[10 * n:11 * n] = -10.0
    f2, m2, v2, n2 = O.densify_prune(flat, m, v, np.ones(n, np.float32), n, np.float32(-5.0), 4)
    assert n2 == 0 and f2.size == 0
    flat[10 * n + 3] = 0.0                          # one survivor with the smallest gradient
    g = np.arange(n, dtype=np.float32)
    f2, m2, v2, n2 = O.densify_prune(flat, m, v, g, n, np.float32(-5.0), 4)
    # kept {3}; clones {3} (pruned ones never cloned); 1 + 1 = 2 -> 2 pads
    assert n2 == 4
    lg = f2[10 * n2:11 * n2]
    assert lg[0] == lg[1] == 0.0 and lg[2] == lg[3] == -30.0


def test_screen_grad_norm_by_hand():
    """Two views, two Gaussians: 3-4-5 and 5-12-13 right triangles; entries
    other than 0 and 1 of a record do not count."""
    g = np.zeros((2, 2, 12))
    g[0, 0, :2] = (3, 4)
    g[1, 0, :2] = (-5, 12)
    g[0, 1, :2] = (0, -2)
    g[:, :, 2:] = 7.0
    assert np.allclose(O.screen_grad_norm(g.ravel(), 2, 2), [5 + 13, 2])


# -- workload-sensitive density control (Sec. III-C) -------------------------

def _line_points():
    # binary-exact coordinates: distances 0.125, 0.25, 0.75, 0.875 are exact
    return np.array([[0.0, 0, 0], [0.125, 0, 0], [0.25, 0, 0], [1.0, 0, 0]], np.float32)


def test_density_stats_on_a_line_by_hand():
    rho, dbar, nn, dnn = O.density_stats(_line_points(), r=0.2, k=2)
    assert rho.tolist() == [1, 2, 1, 0]
    assert dbar.tolist() == [0.1875, 0.125, 0.1875, 0.8125]
    assert nn.tolist() == [1, 0, 1, 2]                 # point 1: two at 0.125, the lower index wins
    assert dnn.tolist() == [0.125, 0.125, 0.125, 0.75]


def test_density_thresholds_closed_form():
    rho = np.array([1, 2, 1, 0])
    dnn = np.array([0.125, 0.125, 0.125, 0.75], np.float32)
    lo, hi, dm = O.density_thresholds(rho, dnn, alpha=1.0, beta=2.0, gamma=0.5)
    sd = np.sqrt(6 / 4 - 1.0)
    assert np.isclose(lo, 1 - sd, rtol=0, atol=1e-15) and np.isclose(hi, 1 + 2 * sd, rtol=0, atol=1e-15)
    mu_d = 1.125 / 4
    sd_d = np.sqrt((3 * 0.125 ** 2 + 0.75 ** 2) / 4 - mu_d ** 2)
    assert np.isclose(dm, mu_d + 0.5 * sd_d, rtol=0, atol=1e-15)


def test_density_stats_on_a_cubic_lattice():
    a = 0.5
    g = np.arange(5, dtype=np.float32) * np.float32(a)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    rho, dbar, nn, dnn = O.density_stats(P, r=0.6, k=6)
    idx = np.arange(125).reshape(5, 5, 5)
    inner = idx[1:4, 1:4, 1:4].ravel()
    assert np.all(rho[inner] == 6)                     # the six face neighbours
    assert np.all(dbar[inner] == np.float32(a))
    corner = idx[0, 0, 0]
    assert rho[corner] == 3
    assert np.all(dnn == np.float32(a))


def _two_clusters(n_dense=40, n_far=6, seed=0, n_core=20):
    """A tight core inside a looser cluster (high densities there) and a few
    far, isolated points (density 0)."""
    rng = np.random.default_rng(seed)
    core = rng.normal(0.0, 0.003, (n_core, 3))
    dense = rng.normal(0.0, 0.02, (n_dense, 3))
    far = rng.uniform(-1, 1, (n_far, 3)) + np.array([3.0, 0, 0])
    return np.concatenate([core, dense, far]).astype(np.float32)


def test_density_control_formulas_by_hand():
    P = _two_clusters()
    n = len(P)
    rng = np.random.default_rng(1)
    flat = rng.normal(0, 1, 59 * n).astype(np.float32)
    flat[:3 * n] = P.ravel()
    m = rng.normal(0, 1, 59 * n).astype(np.float32)
    v = rng.random(59 * n).astype(np.float32)
    z = rng.normal(0, 1, (n, 3)).astype(np.float32)
    u = rng.random((n, 3)).astype(np.float32)
    r, k, ad, delta = 0.03, 3, 1.5, 0.01
    p2, m2, v2, n2, info = O.density_control(flat, m, v, n, r, k, 1.0, 1.0, ad, delta, 1.0, z, u)
    # every far point is alone within r: rho 0 < rho_low, so each spawns one point
    assert info["low"][60:].all() and info["n_new"] >= 6
    assert info["n_merged"] > 0
    assert n2 == info["n_keep"] + info["n_merged"] + info["n_new"] + info["pad"] and n2 % 4 == 0
    G = lambda a, cnt: np.split(a, np.cumsum([3 * cnt, 3 * cnt, 4 * cnt, cnt]))
    out = G(p2, n2)
    mo, vo = G(m2, n2), G(v2, n2)
    means2 = out[0].reshape(n2, 3)
    # untouched points come first, unchanged, with their moments
    keep = np.flatnonzero(~(info["head"] | info["gone"]))
    assert np.array_equal(means2[:len(keep)], P[keep])
    assert np.array_equal(mo[4].reshape(n2, 48)[:len(keep)], m[11 * n:].reshape(n, 48)[keep])
    # merged points: opacity-weighted centroid, log of the mean scale, zero moments
    heads = np.flatnonzero(info["head"])
    i = heads[0]
    j = int(info["nn"][i])
    lg = flat[10 * n:11 * n].astype(np.float64)
    w = 1 / (1 + np.exp(-lg))
    want = (w[i] * P[i] + w[j] * P[j]) / (w[i] + w[j])
    got = means2[len(keep)]
    assert np.allclose(got, want, rtol=0, atol=1e-6)
    ls = flat[3 * n:6 * n].reshape(n, 3).astype(np.float64)
    assert np.allclose(out[1].reshape(n2, 3)[len(keep)], np.log((np.exp(ls[i]) + np.exp(ls[j])) / 2), atol=1e-6)
    better = i if lg[i] >= lg[j] else j
    assert np.array_equal(out[4].reshape(n2, 48)[len(keep)], flat[11 * n:].reshape(n, 48)[better])
    assert not mo[0].reshape(n2, 3)[len(keep)].any()
    # new points: p + alpha_d dbar z + delta (2u - 1), the rest copied from the parent
    first_new = len(keep) + len(heads)
    lows = np.flatnonzero(info["low"])
    a = lows[0]
    want = P[a].astype(np.float64) + ad * float(info["dbar"][a]) * z[a] + delta * (2.0 * u[a] - 1.0)
    assert np.allclose(means2[first_new], want, rtol=0, atol=1e-6)
    assert np.array_equal(out[4].reshape(n2, 48)[first_new], flat[11 * n:].reshape(n, 48)[a])
    # padding: invisible copies
    if info["pad"]:
        assert out[3][-1] == np.float32(-30.0)


def test_density_control_merges_only_mutual_pairs_in_dense_regions():
    P = _two_clusters(60, 4, seed=3)
    n = len(P)
    flat = np.zeros(59 * n, np.float32)
    flat[:3 * n] = P.ravel()
    z = np.zeros((n, 3), np.float32)
    u = np.full((n, 3), 0.5, np.float32)
    _, _, _, n2, info = O.density_control(flat, flat * 0, flat * 0, n, 0.03, 3, 1.0, 1.0, 1.5, 0.0, 1.0, z, u)
    assert info["head"].any() and info["low"].any()
    for i in np.flatnonzero(info["head"]):
        j = info["nn"][i]
        assert info["nn"][j] == i and info["high"][i] and info["high"][j] and j > i
        assert info["dnn"][i] <= info["d_merge"]
    assert not (info["head"] & info["gone"]).any()
    assert not (info["low"] & (info["head"] | info["gone"])).any()


# -- colour hashing (Sec. IV-C1) ---------------------------------------------

def test_colour_quantisation_matches_the_formula_and_bounds():
    c8 = np.arange(256)
    rgb = np.stack([c8, c8, c8], -1).astype(np.float32) / np.float32(255.0)
    h = O.colour_bucket(rgb)
    q = c8 >> 4                                          # floor(c / 256 * 16) for 8-bit c
    assert np.array_equal(h, q * 256 + q * 16 + q)
    assert O.colour_bucket(np.array([1.0, 1.0, 1.0], np.float32)) == 4095      # c = 255 -> 15
    assert O.colour_bucket(np.array([0.0, 0.0, 0.0], np.float32)) == 0
    assert O.colour_bucket(np.array([2.0, -1.0, 0.5], np.float32)) == 15 * 256 + 0 + 8   # clamped; 0.5 -> 128 -> 8
    rng = np.random.default_rng(0)
    hh = O.colour_bucket(rng.uniform(-0.5, 1.5, (10000, 3)).astype(np.float32))
    assert hh.min() >= 0 and hh.max() <= 4095


def test_colour_buckets_by_hand():
    rgb = np.array([[1.0, 0.0, 0.0], [0.99, 0.01, 0.02], [0.0, 0.0, 1.0]], np.float32)
    lo = np.array([-1.0, -2.0, 0.0], np.float32)        # opacities 0.5, 0.25, 1
    ranges = np.array([[0, 3], [3, 3], [3, 5]])
    vals = np.array([0, 1, 2, 1, 1])
    count, sums, distinct = O.colour_buckets(ranges, vals, rgb, lo)
    red, blue = 15 * 256, 15
    assert count[red] == 4 and count[blue] == 1 and count.sum() == 5
    assert np.isclose(sums[0, red], 1.0 + 3 * 0.99) and np.isclose(sums[3, red], 0.5 + 3 * 0.25)
    assert np.isclose(sums[3, blue], 1.0)
    assert distinct.tolist() == [2, 0, 1]


def test_density_point_agrees_with_the_full_statistics():
    """The per-point form used for sampled checks of large inputs gives the
    rows of the all-points form, including ties and the nearest index."""
    P = np.concatenate([_two_clusters(30, 5, seed=7), _line_points()])
    P = np.concatenate([P, P[:4]])                        # exact duplicates: zero distances, ties
    rho, dbar, nn, dnn = O.density_stats(P, r=0.03, k=4)
    for i in (0, 3, 17, 33, 50, 55, len(P) - 1):
        assert O.density_point(P, i, 0.03, 4) == (rho[i], dbar[i], nn[i], dnn[i])


# -- 16-bit storage of the precision path (SH and colours in BF16 / FP16) -----

def _bf16_grid():
    """Every finite non-negative BF16 value, by enumerating bit patterns (a
    BF16 value is a binary32 value whose low 16 bits are zero), ascending,
    with the pattern of each."""
    bits = np.arange(0, 0x7F80, dtype=np.uint32)
    return (bits << np.uint32(16)).view(np.float32).astype(np.float64), bits


def _nearest_even_on_grid(x, grid, bits):
    """Brute-force rounding to a sorted grid: the nearer neighbour, on a tie
    the one whose pattern is even."""
    i = np.clip(np.searchsorted(grid, x), 1, len(grid) - 1)
    lo, hi = grid[i - 1], grid[i]
    dlo, dhi = x - lo, hi - x
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (bits[i] % 2 == 0))
    return np.where(pick_hi, hi, lo)


def test_bf16_rounding_against_brute_force_on_the_whole_grid():
    grid, bits = _bf16_grid()
    rng = np.random.default_rng(0)
    x = np.concatenate([
        np.exp(rng.uniform(np.log(1e-40), np.log(3e38), 200_000)),     # every binade, subnormals too
        rng.uniform(0.0, 4.0, 100_000),                                 # colours and SH
        (grid[1:-1] + grid[2:]) / 2,                                    # every exact midpoint: ties
    ])
    x = x[x < grid[-1]]
    want = _nearest_even_on_grid(x, grid, bits)
    assert np.array_equal(O.round_storage(x, "bf16"), want)
    assert np.array_equal(O.round_storage(-x, "bf16"), -want)          # symmetric
    assert np.array_equal(O.round_storage(grid, "bf16"), grid)         # representable values stay


def test_bf16_rounding_by_hand():
    r = lambda v: float(O.round_storage(v, "bf16"))
    assert r(1.0 + 2.0 ** -8) == 1.0                    # tie, 1.0 has the even significand
    assert r(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # tie, rounds up to the even one
    assert r(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7   # just past the tie
    assert r(0.5 - 2.0 ** -11) == 0.5                   # rounds up across a power of two
    assert r(3.5e38) == math.inf and r(-3.5e38) == -math.inf
    assert r(0.0) == 0.0 and math.isnan(r(math.nan))


def test_f16_rounding_matches_numpy_half():
    rng = np.random.default_rng(1)
    h = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)   # every finite half
    x = np.concatenate([
        np.exp(rng.uniform(np.log(1e-9), np.log(7e4), 200_000)),
        rng.uniform(0.0, 4.0, 100_000),
        (h[1:-1] + h[2:]) / 2,                                          # ties
        [65519.0, 65520.0, 65535.0, 1e5],                               # around overflow
    ])
    x = np.concatenate([x, -x])
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(O.round_storage(x, "f16"), want)
    assert float(O.round_storage(1.0 + 2.0 ** -11, "f16")) == 1.0      # tie to even
    assert float(O.round_storage(65520.0, "f16")) == math.inf


# -- similarity-based sampling and merging of tile lists (Sec. IV-C1) ----------

def test_render_lists_with_the_oracle_lists_is_render():
    """Blending explicit tile lists that are the oracle's own lists, with each
    Gaussian's attributes, gives render() bit for bit."""
    scene = S.uniform_scene(400, 2)
    cam = S.front_camera(96, 64)
    r = O.forward(cam, scene)
    ranges, ids = [], []
    for t in range(cam.n_tiles):
        lst = O.tile_list(r["kp"], t % cam.tiles_x, t // cam.tiles_x)
        ranges.append((len(ids), len(ids) + len(lst)))
        ids.extend(lst.tolist())
    rl = O.render_lists(cam, ranges, np.asarray(ids, np.uint32), r["proj"])
    for k in ("img", "T_final", "n_proc", "flag"):
        assert np.array_equal(rl[k], r[k]), k


def test_colour_merge_by_hand():
    # tile 0: red (0.9, 0.1, 0.1) and red (0.92, 0.08, 0.11) share bucket
    # (14, 1, 1); blue is alone; tile 1: the second red only
    rgb = np.array([[0.9, 0.1, 0.1], [0.2, 0.3, 0.95], [0.92, 0.08, 0.11]], np.float32)
    sp = dict(mean2d=np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]]),
              conic=np.array([[1.0, 0.1, 2.0], [3.0, 0.2, 4.0], [5.0, 0.3, 6.0]]),
              opac=np.array([0.7, 0.4, 0.6]))
    ranges = np.array([[0, 3], [3, 4], [4, 4]])
    vals = np.array([0, 1, 2, 2])
    out_r, ids, reps, src, members = O.colour_merge(ranges, vals, rgb, sp)
    assert out_r.tolist() == [[0, 2], [2, 3], [3, 3]]
    assert src.tolist() == [0, 1, 2] and members.tolist() == [2, 1, 1]
    assert np.allclose(reps["rgb"][0], (rgb[0].astype(np.float64) + rgb[2]) / 2)
    assert reps["opac"][0] == 1.0                     # 0.7 + 0.6, accumulated and capped
    assert reps["opac"][1] == 0.4 and reps["opac"][2] == 0.6
    assert np.array_equal(reps["mean2d"][0], sp["mean2d"][0])       # the first member's place
    assert np.array_equal(reps["conic"][2], sp["conic"][2])


def test_colour_merge_of_two_coincident_splats_closed_form():
    """Two coincident isotropic splats of one colour merge into one of
    opacity min(1, 2 o): at the centre the pixel is min(0.99, 2 o) c, where
    the exact blend gives c (a + a (1 - a)), a = o."""
    cam = S.front_camera(32, 32)
    c, o, s2 = 0.6, 0.3, 9.0
    sp = dict(mean2d=np.array([[16.5, 16.5], [16.5, 16.5]]),
              conic=np.array([[1 / s2, 0.0, 1 / s2]] * 2), opac=np.array([o, o]))
    rgb = np.array([[c, c, c], [c, c, c]], np.float32)
    ranges = np.zeros((cam.n_tiles, 2), np.int64)
    t = (16 // 16) * cam.tiles_x + 16 // 16
    ranges[t:] = 2
    ranges[t, 0] = 0
    out_r, ids, reps, src, members = O.colour_merge(ranges, np.array([0, 1]), rgb, sp)
    assert members.tolist() == [2] and reps["opac"][0] == 2 * o
    m = O.render_lists(cam, out_r, ids, dict(reps, rgb=reps["rgb"]))
    e = O.render_lists(cam, ranges, np.array([0, 1], np.uint32), dict(sp, rgb=rgb.astype(np.float64)))
    cf = float(np.float32(c))
    assert m["img"][0, 16, 16] == pytest.approx(min(0.99, 2 * o) * cf, rel=1e-12)
    assert e["img"][0, 16, 16] == pytest.approx(cf * (o + o * (1 - o)), rel=1e-12)
    # a pixel 2 sigma away: alpha = 2 o exp(-2)
    assert m["img"][0, 16, 22] == pytest.approx(2 * o * math.exp(-0.5 * 36 / s2) * cf, rel=1e-12)


# -- reverse-pass cost features (a8) ------------------------------------------

def test_bwd_tile_features_by_hand():
    cam = S.front_camera(20, 18)                       # 2 x 2 tiles, ragged: 16x16, 4x16, 16x2, 4x2
    n_proc = np.zeros((18, 20), np.int32)
    n_proc[:16, :16] = 3
    n_proc[:16, 16:] = 8
    n_proc[16:, :16] = 0
    n_proc[16:, 16:] = 5
    n_proc[12, 2] = 9                                  # tile 0's lower half holds its deepest pixel
    tile_nproc = np.array([9, 8, 0, 5])
    tile_ns = np.array([1000, 0, 7, 30], np.uint64)
    kept = np.array([40, 12, 0, 3])
    f = O.bwd_tile_features(cam, n_proc, tile_nproc, tile_ns, kept)
    assert np.allclose(f[:, 0], np.log1p([9, 8, 0, 5]))
    assert np.allclose(f[:, 1], np.log1p([3 + 6 / 256, 8, 0, 5]))
    assert np.allclose(f[:, 2], np.log1p([1000, 0, 7, 30]))
    assert np.allclose(f[:, 3], np.log1p([40, 12, 0, 3]))
    # halves: tile 0 (3, 9), tile 1 (8, 8), tile 2 (0, -) and tile 3 (5, -) have no lower half
    assert np.allclose(f[:, 4], np.log1p([6.0, 8.0, 0.0, 2.5]))
    assert np.allclose(f[:, 5], [1.0, 1.0, 0.0, 1.0])
    assert np.allclose(f[:, 6], [1.0, 64 / 256, 32 / 256, 8 / 256])
    assert np.allclose(f[:, 7], math.log1p(360) / 16)

"""TEST INFRASTRUCTURE ONLY: ctypes binding of the CPU oracle (gs_oracle.c).

Only tests/, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import this module.  It never touches the CUDA library.

Conventions: parameters arrive as the float32 arrays of a scene; the FP32
specification path takes them as they are, the FP64 path takes them widened
to float64 (exact).  Images are [3, H, W]; per-pixel maps are [H, W].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "gs_oracle.c"
BUILD_DIR = HERE / "_build"
LIB_PATH = BUILD_DIR / "libgs_oracle.so"

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc: -O2, IEEE arithmetic, no FP contraction."""
    BUILD_DIR.mkdir(exist_ok=True)
    if not force and LIB_PATH.exists() and LIB_PATH.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB_PATH
    tmp = LIB_PATH.with_suffix(f".so.tmp{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", str(tmp), str(SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrcCam(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("campos", ctypes.c_float * 3), ("znear", ctypes.c_float),
                ("bg", ctypes.c_float * 3)]


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


F32 = ctypes.c_float
F64 = ctypes.c_double
I32 = ctypes.c_int
U32 = ctypes.c_uint
I64 = ctypes.c_longlong
U8 = ctypes.c_ubyte


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB_PATH))
        P = ctypes.POINTER
        L.orc_exp_spec.restype = F32
        L.orc_exp_spec.argtypes = [F32]
        L.orc_keypath_f32.argtypes = [P(OrcCam), I32, P(F32), P(F32), P(F32), P(F32), P(F32),
                                      P(F32), P(I32), P(I32), P(I32), P(I32)]
        L.orc_tile_list.restype = I64
        L.orc_tile_list.argtypes = [I32, P(I32), P(I32), P(F32), I32, I32, P(U32), I64]
        L.orc_tile_counts.argtypes = [P(OrcCam), I32, P(I32), P(I32), P(I64)]
        L.orc_sh_basis.argtypes = [F64, F64, F64, P(F64), P(F64)]
        L.orc_project_f64.argtypes = [P(OrcCam), I32] + [P(F64)] * 5 + [P(I32)] + [P(F64)] * 5
        L.orc_render_fwd.restype = I64
        L.orc_render_fwd.argtypes = ([P(OrcCam), I32, P(I32), P(I32), P(F32)] + [P(F64)] * 4 +
                                     [I32] * 4 + [F64, F64, P(F64), P(F64), P(I32), P(U8)])
        L.orc_render_lists.restype = I64
        L.orc_render_lists.argtypes = ([P(OrcCam), P(I64), P(U32)] + [P(F64)] * 4 + [I32] * 4 +
                                       [F64, F64, P(F64), P(F64), P(I32), P(U8)])
        L.orc_render_bwd.argtypes = ([P(OrcCam), I32, P(I32), P(I32), P(F32)] + [P(F64)] * 4 +
                                     [I32] * 4 + [P(F64), P(F64)])
        L.orc_project_bwd.argtypes = [P(OrcCam), I32] + [P(F64)] * 5 + [P(I32), P(F64), P(F64)]
        L.orc_l1.restype = F64
        L.orc_l1.argtypes = [I64, P(F64), P(F64), P(F64)]
        L.orc_adam.argtypes = [I64, P(F64), P(F64), P(F64), P(F64), P(F64), F64, F64, F64, I32]
        L.orc_mlp_fwd.argtypes = [I32] + [P(F64)] * 6
        L.orc_mlp_loss_grad.restype = F64
        L.orc_mlp_loss_grad.argtypes = [I32] + [P(F64)] * 7
        L.orc_tile_features.argtypes = [P(OrcCam), I32, P(I32), P(I32), P(F32), P(F64), P(F64),
                                        I32, I32, I64, P(F64)]
        L.orc_set_threads.argtypes = [I32]
        L.orc_get_threads.restype = I32
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def cam_struct(cam) -> OrcCam:
    c = OrcCam()
    c.W, c.H = int(cam.W), int(cam.H)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    for k, v in enumerate(np.asarray(cam.R, np.float32).ravel()):
        c.R[k] = float(v)
    for k, v in enumerate(np.asarray(cam.t, np.float32).ravel()):
        c.t[k] = float(v)
    for k, v in enumerate(np.asarray(cam.campos, np.float32).ravel()):
        c.campos[k] = float(v)
    c.znear = float(cam.znear)
    for k, v in enumerate(cam.bg):
        c.bg[k] = float(v)
    return c


def exp_spec(x: float) -> float:
    return float(lib().orc_exp_spec(float(x)))


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def keypath(cam, scene) -> dict:
    """FP32 specification path: depth, mean2d, cov2d, radius, rect, touched."""
    n = scene.n
    means, ls, q = _c32(scene.means), _c32(scene.log_scales), _c32(scene.quats)
    out = dict(depth=np.zeros(n, np.float32), mean2d=np.zeros((n, 2), np.float32),
               cov2d=np.zeros((n, 3), np.float32), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), touched=np.zeros(n, np.int32),
               status=np.zeros(n, np.int32))
    c = cam_struct(cam)
    lib().orc_keypath_f32(ctypes.byref(c), n, _p(means, F32), _p(ls, F32), _p(q, F32),
                          _p(out["depth"], F32), _p(out["mean2d"], F32), _p(out["cov2d"], F32),
                          _p(out["radius"], I32), _p(out["rect"], I32), _p(out["touched"], I32),
                          _p(out["status"], I32))
    return out


def tile_list(kp: dict, tx: int, ty: int) -> np.ndarray:
    n = kp["depth"].shape[0]
    L = lib()
    cnt = L.orc_tile_list(n, _p(kp["rect"], I32), _p(kp["touched"], I32), _p(kp["depth"], F32),
                          tx, ty, None, 0)
    ids = np.zeros(max(cnt, 1), np.uint32)
    L.orc_tile_list(n, _p(kp["rect"], I32), _p(kp["touched"], I32), _p(kp["depth"], F32),
                    tx, ty, _p(ids, U32), cnt)
    return ids[:cnt]


def tile_counts(cam, kp: dict) -> np.ndarray:
    c = cam_struct(cam)
    out = np.zeros(cam.n_tiles, np.int64)
    lib().orc_tile_counts(ctypes.byref(c), kp["depth"].shape[0], _p(kp["rect"], I32),
                          _p(kp["touched"], I32), _p(out, I64))
    return out


def sh_basis(x: float, y: float, z: float):
    Y = np.zeros(16, np.float64)
    G = np.zeros((16, 3), np.float64)
    lib().orc_sh_basis(float(x), float(y), float(z), _p(Y, F64), _p(G, F64))
    return Y, G


def project(cam, scene, kp: dict, params64: dict | None = None) -> dict:
    """FP64 projection.  params64 overrides the scene's parameters (float64
    arrays with keys means, log_scales, quats, opacity_logits, sh)."""
    n = scene.n
    p = params64 or {}
    means = _c64(p.get("means", scene.means))
    ls = _c64(p.get("log_scales", scene.log_scales))
    q = _c64(p.get("quats", scene.quats))
    lg = _c64(p.get("opacity_logits", scene.opacity_logits))
    sh = _c64(p.get("sh", scene.sh)).reshape(n, 48)
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opac=np.zeros(n),
               rgb=np.zeros((n, 3)), rgb_pre=np.zeros((n, 3)))
    c = cam_struct(cam)
    lib().orc_project_f64(ctypes.byref(c), n, _p(means, F64), _p(ls, F64), _p(q, F64),
                          _p(lg, F64), _p(sh, F64), _p(kp["touched"], I32),
                          _p(out["mean2d"], F64), _p(out["conic"], F64), _p(out["opac"], F64),
                          _p(out["rgb"], F64), _p(out["rgb_pre"], F64))
    return out


def _window(cam, window):
    if window is None:
        return 0, 0, cam.W, cam.H
    return tuple(int(v) for v in window)


def render(cam, kp: dict, proj: dict, window=None, margin_alpha: float = 1e-4,
           margin_T: float = 1e-3) -> dict:
    """FP64 forward blend over the pixel window (x0, y0, x1, y1)."""
    x0, y0, x1, y1 = _window(cam, window)
    n = kp["depth"].shape[0]
    W, H = cam.W, cam.H
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nproc = np.zeros((H, W), np.int32)
    flag = np.zeros((H, W), np.uint8)
    c = cam_struct(cam)
    m2, co, op, rgb = (_c64(proj[k]) for k in ("mean2d", "conic", "opac", "rgb"))
    pairs = lib().orc_render_fwd(ctypes.byref(c), n, _p(kp["rect"], I32), _p(kp["touched"], I32),
                                 _p(kp["depth"], F32), _p(m2, F64), _p(co, F64), _p(op, F64),
                                 _p(rgb, F64), x0, y0, x1, y1, margin_alpha, margin_T,
                                 _p(img, F64), _p(T, F64), _p(nproc, I32), _p(flag, U8))
    return dict(img=img, T_final=T, n_proc=nproc, flag=flag, pairs=int(pairs))


def render_lists(cam, ranges, ids, splats: dict, window=None, margin_alpha: float = 1e-4,
                 margin_T: float = 1e-3) -> dict:
    """FP64 forward blend of the pixel window from explicit tile lists: tile t
    (row-major) blends splats ids[ranges[t, 0]:ranges[t, 1]] in that order
    (splats: mean2d [m, 2], conic [m, 3], opac [m], rgb [m, 3]), with the
    per-pixel rules of render()."""
    x0, y0, x1, y1 = _window(cam, window)
    W, H = cam.W, cam.H
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nproc = np.zeros((H, W), np.int32)
    flag = np.zeros((H, W), np.uint8)
    rg = np.ascontiguousarray(np.asarray(ranges, np.int64).reshape(-1, 2))
    idv = np.ascontiguousarray(np.asarray(ids, np.uint32))
    if idv.size == 0:
        idv = np.zeros(1, np.uint32)
    m2, co, op, rgb = (_c64(splats[k]) for k in ("mean2d", "conic", "opac", "rgb"))
    c = cam_struct(cam)
    pairs = lib().orc_render_lists(ctypes.byref(c), _p(rg, I64), _p(idv, U32), _p(m2, F64), _p(co, F64),
                                   _p(op, F64), _p(rgb, F64), x0, y0, x1, y1, margin_alpha, margin_T,
                                   _p(img, F64), _p(T, F64), _p(nproc, I32), _p(flag, U8))
    return dict(img=img, T_final=T, n_proc=nproc, flag=flag, pairs=int(pairs))


def render_bwd(cam, kp: dict, proj: dict, dL_dimg: np.ndarray, window=None) -> np.ndarray:
    """Gradient with respect to (u, v, A, B, C, opacity, r, g, b) per Gaussian."""
    x0, y0, x1, y1 = _window(cam, window)
    n = kp["depth"].shape[0]
    g = np.zeros((n, 9))
    c = cam_struct(cam)
    m2, co, op, rgb = (_c64(proj[k]) for k in ("mean2d", "conic", "opac", "rgb"))
    d = _c64(dL_dimg)
    lib().orc_render_bwd(ctypes.byref(c), n, _p(kp["rect"], I32), _p(kp["touched"], I32),
                         _p(kp["depth"], F32), _p(m2, F64), _p(co, F64), _p(op, F64), _p(rgb, F64),
                         x0, y0, x1, y1, _p(d, F64), _p(g, F64))
    return g


def project_bwd(cam, scene, kp: dict, grad2d: np.ndarray, params64: dict | None = None) -> np.ndarray:
    """Gradient of the 59 parameters, grouped [means|log_scales|quats|logits|sh]."""
    n = scene.n
    p = params64 or {}
    means = _c64(p.get("means", scene.means))
    ls = _c64(p.get("log_scales", scene.log_scales))
    q = _c64(p.get("quats", scene.quats))
    lg = _c64(p.get("opacity_logits", scene.opacity_logits))
    sh = _c64(p.get("sh", scene.sh)).reshape(n, 48)
    out = np.zeros(59 * n)
    g2 = _c64(grad2d)
    c = cam_struct(cam)
    lib().orc_project_bwd(ctypes.byref(c), n, _p(means, F64), _p(ls, F64), _p(q, F64),
                          _p(lg, F64), _p(sh, F64), _p(kp["touched"], I32), _p(g2, F64),
                          _p(out, F64))
    return out


def split_params(flat: np.ndarray, n: int) -> dict:
    """View a grouped 59 n buffer as its named parameter groups."""
    o = 0
    out = {}
    for name, w in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)):
        out[name] = flat[o:o + w * n].reshape((n, w) if w > 1 else (n,))
        o += w * n
    out["sh"] = out["sh"].reshape(n, 16, 3)
    return out


def l1(img: np.ndarray, tgt: np.ndarray):
    a, b = _c64(img).ravel(), _c64(tgt).ravel()
    d = np.zeros_like(a)
    loss = lib().orc_l1(a.size, _p(a, F64), _p(b, F64), _p(d, F64))
    return float(loss), d.reshape(np.shape(img))


def adam(p, g, m, v, lr, b1=0.9, b2=0.999, eps=1e-15, step=1):
    """One Adam step in FP64; returns new (p, m, v).  lr is per entry."""
    p, g, m, v = (_c64(x).copy() for x in (p, g, m, v))
    lr = _c64(np.broadcast_to(lr, p.shape))
    lib().orc_adam(p.size, _p(p, F64), _p(g, F64), _p(m, F64), _p(v, F64), _p(lr, F64),
                   b1, b2, eps, int(step))
    return p, m, v


def mlp_fwd(feats, W1, b1, W2, b2) -> np.ndarray:
    f = _c64(feats)
    n = f.shape[0]
    y = np.zeros(n)
    lib().orc_mlp_fwd(n, _p(f, F64), _p(_c64(W1), F64), _p(_c64(b1), F64), _p(_c64(W2), F64),
                      _p(_c64(np.atleast_1d(b2)), F64), _p(y, F64))
    return y


def mlp_loss_grad(feats, target, W1, b1, W2, b2):
    f = _c64(feats)
    n = f.shape[0]
    g = np.zeros(321)
    loss = lib().orc_mlp_loss_grad(n, _p(f, F64), _p(_c64(target), F64), _p(_c64(W1), F64),
                                   _p(_c64(b1), F64), _p(_c64(W2), F64),
                                   _p(_c64(np.atleast_1d(b2)), F64), _p(g, F64))
    return float(loss), g


def tile_features(cam, kp: dict, proj: dict, tx: int, ty: int, cap: int = 4096) -> np.ndarray:
    """The eight per-tile cost features of tile (tx, ty)."""
    n = kp["depth"].shape[0]
    cov = proj["conic"]
    # det of the dilated Sigma' from its inverse: det(Sigma') = 1 / det(conic)
    dconic = cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2
    det = np.where(dconic > 0, 1.0 / np.where(dconic > 0, dconic, 1.0), 0.0)
    f = np.zeros(8)
    c = cam_struct(cam)
    lib().orc_tile_features(ctypes.byref(c), n, _p(kp["rect"], I32), _p(kp["touched"], I32),
                            _p(kp["depth"], F32), _p(_c64(proj["opac"]), F64), _p(_c64(det), F64),
                            tx, ty, cap, _p(f, F64))
    return f


def bwd_tile_features(cam, n_proc, tile_nproc, tile_ns, kept) -> np.ndarray:
    """The reverse pass's eight cost features of every tile of one view
    ([n_tiles, 8], FP64), from what the forward pass left: b0 log1p(the
    tile's largest processed count), b1 log1p(mean processed count over its
    in-image pixels), b2 log1p(the forward's time of the tile, ns), b3
    log1p(its kept list length), b4 log1p(mean over its upper and lower
    16x8 halves of their largest processed count), b5 the fraction of its
    in-image pixels with a processed count > 0, b6 the in-image pixel
    fraction, b7 log1p(W H) / 16.  n_proc is the [H, W] map of processed
    counts."""
    npm = np.maximum(np.asarray(n_proc, np.float64).reshape(cam.H, cam.W), 0)
    out = np.zeros((cam.n_tiles, 8))
    for t in range(cam.n_tiles):
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        block = npm[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16]
        top, bottom = block[:8], block[8:]
        halves = [h.max() if h.size else 0.0 for h in (top, bottom)]
        out[t, 0] = np.log1p(max(0, int(tile_nproc[t])))
        out[t, 1] = np.log1p(block.sum() / block.size)
        out[t, 2] = np.log1p(float(tile_ns[t]))
        out[t, 3] = np.log1p(float(kept[t]))
        out[t, 4] = np.log1p(0.5 * (halves[0] + halves[1]))
        out[t, 5] = (block > 0).sum() / block.size
        out[t, 6] = block.size / 256.0
        out[t, 7] = np.log1p(float(cam.W) * cam.H) / 16.0
    return out


def forward(cam, scene, window=None, margin_alpha=1e-4, margin_T=1e-3) -> dict:
    """Key path + FP64 projection + render, in one call."""
    kp = keypath(cam, scene)
    proj = project(cam, scene, kp)
    r = render(cam, kp, proj, window, margin_alpha, margin_T)
    r.update(kp=kp, proj=proj)
    return r


# 16-bit storage formats of the precision path (SH coefficients and colours
# stored in BF16 or FP16, everything computed from them in wider precision):
# (significand bits including the implicit one, minimum normal exponent,
# largest finite value).
STORAGE_FORMATS = {
    "bf16": (8, -126, (2.0 - 2.0 ** -7) * 2.0 ** 127),
    "f16": (11, -14, 65504.0),
}


def round_storage(x, kind: str) -> np.ndarray:
    """The value a 16-bit storage format holds for x: the nearest value of the
    format, ties to the even significand (IEEE 754 roundTiesToEven), values
    beyond the overflow threshold to infinity; returned as float64.

    Written from the definition of a binary floating-point format with p
    significand bits and minimum exponent emin: below 2^(emin + 1) the
    spacing is the subnormal one, 2^(emin - p + 1); in [2^e, 2^(e + 1)) it is
    2^(e - p + 1).  Dividing by that power of two is exact, np.rint rounds
    half to even, and multiplying back is exact."""
    p, emin, vmax = STORAGE_FORMATS[kind]
    x = np.asarray(x, np.float64)
    _, e = np.frexp(np.abs(x))                 # |x| = m 2^e with m in [0.5, 1)
    ulp = np.ldexp(1.0, np.maximum(e - 1, emin) - (p - 1))
    with np.errstate(invalid="ignore", over="ignore"):
        r = np.rint(x / ulp) * ulp
        r = np.where(np.abs(r) > vmax, np.copysign(np.inf, x), r)
    return np.where(np.isfinite(x), r, x)


def densify_prune(flat, m, v, grad_norm, n, logit_threshold, n_clone):
    """One densification step of dynamic training (density control, Sec. III-B,
    in its plain clone-and-prune form).  Written out from its definition:

    - keep Gaussian i iff its opacity logit >= logit_threshold (FP32 values,
      compared as stored: the threshold is the FP32 logit of the minimum
      opacity);
    - rank the kept Gaussians by screen-space gradient norm g_i, descending,
      ties by index (g_i <= 0 or NaN counts as 0), and clone the first
      c = min(n_clone, kept) of them;
    - the new count must be a multiple of 4 (the grouped layout's alignment):
      drop the last (kept + c) mod 4 clones when there are that many, else pad
      with copies of the first kept Gaussian made invisible (logit -30);
    - output: the kept Gaussians in index order, then the clones in rank
      order, then the pads, in the grouped layout of the new count; clones and
      pads start with zero Adam moments, kept Gaussians keep theirs.

    Returns (flat', m', v', n')."""
    flat, m, v = (np.asarray(a, np.float32) for a in (flat, m, v))
    widths = (3, 3, 4, 1, 48)
    def groups(a, count):
        out, o = [], 0
        for w in widths:
            out.append(a[o:o + w * count].reshape(count, w))
            o += w * count
        return out
    P, M, V = groups(flat, n), groups(m, n), groups(v, n)
    logit = P[3][:, 0]
    keep = np.flatnonzero(logit >= np.float32(logit_threshold))
    g = np.asarray(grad_norm, np.float32)
    g = np.where(g > 0, g, np.float32(0))
    ranked = sorted(keep.tolist(), key=lambda i: (-float(g[i]), i))
    c = min(int(n_clone), len(keep))
    r = (len(keep) + c) % 4
    if r and c >= r:
        c -= r
    clones = ranked[:c]
    pad = (-(len(keep) + c)) % 4 if len(keep) else 0
    src = keep.tolist() + clones + ([int(keep[0])] * pad if pad else [])
    n2 = len(src)
    fresh = np.array([False] * len(keep) + [True] * (c + pad))
    outP, outM, outV = [], [], []
    for gi in range(5):
        pg = P[gi][src].copy() if n2 else np.zeros((0, widths[gi]), np.float32)
        if gi == 3 and pad:
            pg[len(keep) + c:, 0] = np.float32(-30.0)
        mg = M[gi][src].copy() if n2 else np.zeros((0, widths[gi]), np.float32)
        vg = V[gi][src].copy() if n2 else np.zeros((0, widths[gi]), np.float32)
        if n2:
            mg[fresh] = 0.0
            vg[fresh] = 0.0
        outP.append(pg.ravel())
        outM.append(mg.ravel())
        outV.append(vg.ravel())
    return np.concatenate(outP), np.concatenate(outM), np.concatenate(outV), n2


def screen_grad_norm(grad2d, n_views, n):
    """Screen-space gradient statistic that selects the Gaussians to clone
    (adaptive density control, Sec. II-A): for Gaussian i, the sum over views
    of the Euclidean norm of (dL/du, dL/dv), entries 0 and 1 of its record
    (view v, Gaussian i at record v n + i, 12 floats per record)."""
    g = np.asarray(grad2d, np.float64).reshape(n_views, n, 12)
    return np.sqrt(g[:, :, 0] ** 2 + g[:, :, 1] ** 2).sum(axis=0)


# ---------------------------------------------------------------------------
# Workload-sensitive density control (Sec. III-C), written from its
# definitions with brute-force pairwise distances.  Distances are FP32, each
# squared distance summed as (dx^2 + dy^2) + dz^2 with every operation
# rounded (no fused multiply-add), so the integer decisions they feed
# (neighbour counts, nearest neighbours) are reproducible bit for bit.
# ---------------------------------------------------------------------------

def _pair_d2(P, rows):
    """FP32 squared distances from points `rows` to every point, [len(rows), n]."""
    d = [(P[None, :, a] - P[rows, None, a]).astype(np.float32) for a in range(3)]
    return ((d[0] * d[0] + d[1] * d[1]).astype(np.float32) + d[2] * d[2]).astype(np.float32)


def density_stats(means, r, k, chunk=512):
    """Per point: local density rho_p = #{q != p : |q - p| <= r} (Sec. III-C1,
    squared distances against fl32(r) * fl32(r)); the mean distance to the k
    nearest other points, d_bar = (sum of the k smallest distances, ascending,
    in FP32) / k (fewer when fewer points exist, 0 with none, Sec. III-C2); the
    nearest neighbour (ties by index, -1 with none) and its distance."""
    P = np.ascontiguousarray(means, np.float32)
    n = P.shape[0]
    r2 = np.float32(np.float32(r) * np.float32(r))
    rho = np.zeros(n, np.int64)
    dbar = np.zeros(n, np.float32)
    nn = np.full(n, -1, np.int64)
    dnn = np.zeros(n, np.float32)
    kk = min(k, n - 1)
    for a in range(0, n, chunk):
        rows = np.arange(a, min(n, a + chunk))
        d2 = _pair_d2(P, rows)
        d2[np.arange(len(rows)), rows] = np.inf                  # not its own neighbour
        rho[rows] = (d2 <= r2).sum(axis=1)
        if kk <= 0:
            continue
        # the kk smallest by (distance, index): every entry up to the kk-th
        # smallest value is a candidate, ordered by value then index
        kth = np.partition(d2, kk - 1, axis=1)[:, kk - 1]
        order = np.empty((len(rows), kk), np.int64)
        for t in range(len(rows)):
            cand = np.flatnonzero(d2[t] <= kth[t])
            order[t] = cand[np.lexsort((cand, d2[t, cand]))][:kk]
        near = np.sqrt(np.take_along_axis(d2, order, axis=1)).astype(np.float32)
        acc = np.zeros(len(rows), np.float32)
        for j in range(kk):
            acc = (acc + near[:, j]).astype(np.float32)
        dbar[rows] = (acc / np.float32(kk)).astype(np.float32)
        nn[rows] = order[:, 0]
        dnn[rows] = near[:, 0]
    return rho, dbar, nn, dnn


def density_point(means, i, r, k):
    """density_stats for the single point i against every point (for sampled
    checks of large inputs): (rho, d_bar, nearest index, nearest distance)."""
    P = np.ascontiguousarray(means, np.float32)
    d2 = _pair_d2(P, np.array([i]))[0]
    d2[i] = np.inf
    r2 = np.float32(np.float32(r) * np.float32(r))
    kk = min(k, len(P) - 1)
    if kk <= 0:
        return int((d2 <= r2).sum()), np.float32(0), -1, np.float32(0)
    order = np.lexsort((np.arange(len(P)), d2))[:kk]
    near = np.sqrt(d2[order]).astype(np.float32)
    acc = np.float32(0)
    for x in near:
        acc = np.float32(acc + x)
    return int((d2 <= r2).sum()), np.float32(acc / np.float32(kk)), int(order[0]), near[0]


def density_thresholds(rho, dnn, alpha, beta, gamma):
    """rho_low = mu - alpha sigma, rho_high = mu + beta sigma over the local
    densities (Sec. III-C1; population standard deviation), and the merge
    radius d_merge = mu_d + gamma sigma_d over the nearest-neighbour
    distances (Sec. III-C3), in FP64: mu = S1 / n, sigma = sqrt(max(0,
    S2 / n - mu^2)) from exact integer sums for rho."""
    n = len(rho)
    if n == 0:
        return 0.0, 0.0, 0.0
    s1, s2 = int(np.sum(rho)), int(np.sum(rho.astype(object) ** 2))
    mu = float(s1) / n
    var = float(s2) / n - mu * mu
    sd = float(np.sqrt(max(var, 0.0)))
    lo, hi = mu - alpha * sd, mu + beta * sd
    if n < 2:
        return lo, hi, 0.0
    d = dnn.astype(np.float64)
    mu_d = float(d.sum()) / n
    var_d = float((d * d).sum()) / n - mu_d * mu_d
    return lo, hi, mu_d + gamma * float(np.sqrt(max(var_d, 0.0)))


def density_control(flat, m, v, n, r, k, alpha, beta, alpha_d, delta, gamma, z, u):
    """One round of workload-sensitive density control (Sec. III-C).

    - thresholds from the local densities (density_thresholds);
    - every point with rho < rho_low spawns one new point (Sec. III-C2):
      p_new = p + sigma_p z + delta (2 u - 1), sigma_p = alpha_d d_bar_p, with
      the draws z ~ N(0, 1)^3 and u ~ U[0, 1)^3 given; the rest of the new
      Gaussian is a copy of its parent;
    - a point with rho > rho_high merges with its nearest neighbour when the
      two are each other's nearest neighbour, both have rho > rho_high and
      their distance is <= d_merge (Sec. III-C3): position = opacity-weighted
      centroid (weights sigmoid(logit)), log-scale = log of the mean scale per
      axis, every other parameter from the more opaque of the two (larger
      logit, ties to the lower index);
    - output (grouped layout of the new count): the untouched points in index
      order, the merged points in the order of their lower index, the new
      points in the order of their parents, then padding to a multiple of 4
      (copies of output point 0 with logit -30); merged, new and padding
      points start with zero Adam moments.
    Returns (flat', m', v', n', info)."""
    flat, m, v = (np.asarray(a, np.float32) for a in (flat, m, v))
    widths = (3, 3, 4, 1, 48)
    def groups(a, count):
        out, o = [], 0
        for w in widths:
            out.append(a[o:o + w * count].reshape(count, w))
            o += w * count
        return out
    Pg, Mg, Vg = groups(flat, n), groups(m, n), groups(v, n)
    means = Pg[0]
    rho, dbar, nn, dnn = density_stats(means, r, k)
    lo, hi, dm = density_thresholds(rho, dnn, alpha, beta, gamma)
    low = rho.astype(np.float64) < lo
    high = rho.astype(np.float64) > hi
    head = np.zeros(n, bool)
    gone = np.zeros(n, bool)
    for i in range(n):
        j = int(nn[i])
        if j > i and high[i] and high[j] and nn[j] == i and float(dnn[i]) <= dm:
            head[i] = True
            gone[j] = True
    keep = ~(head | gone)
    z, u = np.asarray(z, np.float32), np.asarray(u, np.float32)
    rows = []                      # (parameters, fresh) per output point, group by group
    def point(i):
        return [g[i].copy() for g in Pg]
    for i in np.flatnonzero(keep):
        rows.append(([g[i].copy() for g in Pg], [g[i].copy() for g in Mg], [g[i].copy() for g in Vg]))
    for i in np.flatnonzero(head):
        j = int(nn[i])
        pi, pj = point(i), point(j)
        li, lj = pi[3][0], pj[3][0]
        wi = np.float32(1.0) / (np.float32(1.0) + np.exp(-li, dtype=np.float32))
        wj = np.float32(1.0) / (np.float32(1.0) + np.exp(-lj, dtype=np.float32))
        pos = ((wi * pi[0] + wj * pj[0]) / (wi + wj)).astype(np.float32)
        ls = np.log(np.float32(0.5) * (np.exp(pi[1]) + np.exp(pj[1]))).astype(np.float32)
        src = pi if li >= lj else pj
        q = [pos, ls] + [src[g].copy() for g in (2, 3, 4)]
        rows.append((q, [np.zeros(w, np.float32) for w in widths], [np.zeros(w, np.float32) for w in widths]))
    f32 = np.float32
    for i in np.flatnonzero(low):
        pi = point(i)
        s = f32(f32(alpha_d) * dbar[i])
        jit = (f32(2.0) * u[i] - f32(1.0)).astype(np.float32)
        pos = ((means[i] + (s * z[i]).astype(np.float32)).astype(np.float32)
               + (f32(delta) * jit).astype(np.float32)).astype(np.float32)
        q = [pos] + [pi[g].copy() for g in (1, 2, 3, 4)]
        rows.append((q, [np.zeros(w, np.float32) for w in widths], [np.zeros(w, np.float32) for w in widths]))
    pad = (-len(rows)) % 4 if rows else 0
    for _ in range(pad):
        q = [g.copy() for g in rows[0][0]]
        q[3] = np.array([-30.0], np.float32)
        rows.append((q, [np.zeros(w, np.float32) for w in widths], [np.zeros(w, np.float32) for w in widths]))
    n2 = len(rows)
    outs = []
    for which in range(3):
        parts = [np.stack([row[which][g] for row in rows]).ravel() if n2 else np.zeros(0, np.float32)
                 for g in range(5)]
        outs.append(np.concatenate(parts).astype(np.float32))
    info = dict(rho=rho, dbar=dbar, nn=nn, dnn=dnn, rho_low=lo, rho_high=hi, d_merge=dm,
                low=low, high=high, head=head, gone=gone, n_keep=int(keep.sum()),
                n_merged=int(head.sum()), n_new=int(low.sum()), pad=pad)
    return outs[0], outs[1], outs[2], n2, info


# ---------------------------------------------------------------------------
# Colour hashing of the Gaussians listed per 16x16 tile (Sec. IV-C1).
# ---------------------------------------------------------------------------

def colour_bucket(rgb):
    """Bucket of each colour: every channel to 8 bits as floor(fl32(fl32(c *
    255) + 0.5)) clamped to [0, 255], quantised to c_q = floor(c8 / 256 * 16)
    (16 levels), hash = R_q * 256 + G_q * 16 + B_q in [0, 4095]."""
    c = np.asarray(rgb, np.float32)
    c8 = np.floor((c * np.float32(255.0)).astype(np.float32) + np.float32(0.5)).astype(np.int64)
    c8 = np.clip(c8, 0, 255)
    q = np.floor(c8 / 256.0 * 16.0).astype(np.int64)
    return q[..., 0] * 256 + q[..., 1] * 16 + q[..., 2]


def colour_merge(ranges, vals, record_rgb, splats: dict):
    """Similarity-based sampling and merging of tile lists (Sec. IV-C1), one
    16x16 tile at a time.  A tile's entries are grouped by the bucket of
    their record colour (colour_bucket); each bucket is represented by its
    first entry in list (depth) order, which keeps that Gaussian's position,
    shape and place in the list, and takes the bucket's averaged colour
    (mean of the members' record colours) and accumulated opacity
    min(1, sum of the members' opacities); the other members are dropped.

    ranges [T, 2] and vals: the tile lists; record_rgb [n, 3]: the colour
    each record holds (hashed and averaged); splats: FP64 mean2d, conic,
    opac of the n Gaussians.  Returns (ranges', ids', reps, src, members):
    the merged lists (tile after tile, ids' indexing reps), the
    representatives (mean2d, conic, opac, rgb; FP64), the Gaussian each
    representative stands at and its member count."""
    ranges = np.asarray(ranges, np.int64).reshape(-1, 2)
    vals = np.asarray(vals, np.int64)
    rec = np.asarray(record_rgb, np.float32)
    h_all = colour_bucket(rec)
    rgb64 = rec.astype(np.float64)
    op = np.asarray(splats["opac"], np.float64)
    out_ranges = np.zeros_like(ranges)
    src, members, rgb, opac = [], [], [], []
    for t, (a, b) in enumerate(ranges):
        out_ranges[t, 0] = len(src)
        first = {}                                  # bucket -> representative number
        for g in vals[a:b]:
            h = int(h_all[g])
            if h not in first:
                first[h] = len(src)
                src.append(int(g))
                members.append(0)
                rgb.append(np.zeros(3))
                opac.append(0.0)
            r = first[h]
            members[r] += 1
            rgb[r] = rgb[r] + rgb64[g]
            opac[r] += op[g]
        out_ranges[t, 1] = len(src)
    src = np.asarray(src, np.int64)
    members = np.asarray(members, np.int64)
    reps = dict(mean2d=np.asarray(splats["mean2d"], np.float64)[src].reshape(-1, 2),
                conic=np.asarray(splats["conic"], np.float64)[src].reshape(-1, 3),
                opac=np.minimum(1.0, np.asarray(opac, np.float64)),
                rgb=np.asarray(rgb, np.float64).reshape(-1, 3) / np.maximum(members, 1)[:, None])
    return out_ranges, np.arange(len(src), dtype=np.uint32), reps, src, members


def colour_buckets(ranges, vals, rgb, lo):
    """Bucket-wise aggregation over every tile's list (Sec. IV-C1): per bucket
    the number of (tile, Gaussian) entries, the sums of their colours and of
    their opacities 2^lo (FP64), and per tile the number of distinct buckets
    among its entries."""
    ranges = np.asarray(ranges, np.int64).reshape(-1, 2)
    vals = np.asarray(vals, np.int64)
    h_all = colour_bucket(rgb)
    count = np.zeros(4096, np.int64)
    sums = np.zeros((4, 4096), np.float64)
    distinct = np.zeros(len(ranges), np.int64)
    rgb64 = np.asarray(rgb, np.float32).astype(np.float64)
    op = np.exp2(np.asarray(lo, np.float32).astype(np.float64))
    for t, (a, b) in enumerate(ranges):
        ids = vals[a:b]
        if len(ids) == 0:
            continue
        h = h_all[ids]
        np.add.at(count, h, 1)
        for ch in range(3):
            np.add.at(sums[ch], h, rgb64[ids, ch])
        np.add.at(sums[3], h, op[ids])
        distinct[t] = len(np.unique(h))
    return count, sums, distinct

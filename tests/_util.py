"""Shared helpers of the GPU parity tests: run the CUDA path, decode its
buffers, and compare with the oracle at the stated tolerances."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O
from paper_2510_14564_gb300 import scenes as S

LN2 = math.log(2.0)

# Tolerances (FP32 path against the FP64 oracle)
IMG_ATOL = 1e-4        # image, per channel, unflagged pixels
GRAD_RTOL = 1e-3       # gradients, relative


def decode_splats(splats_f32: np.ndarray, n: int, rgb_dtype: int) -> dict:
    """Host decode of splat records into (u, v, A, B, C, opacity, rgb)."""
    import torch
    if rgb_dtype == 0:
        r = splats_f32.reshape(n, 12)
        rgb = r[:, 6:9].copy()
    else:
        r = splats_f32.reshape(n, 8)
        raw = r[:, 6:8].copy().view(np.uint32)
        lo16 = (raw & 0xFFFF).astype(np.uint16)
        hi16 = (raw >> 16).astype(np.uint16)
        tdt = torch.bfloat16 if rgb_dtype == 1 else torch.float16
        cvt = lambda a: torch.from_numpy(a.view(np.int16).copy()).view(tdt).float().numpy()
        rgb = np.stack([cvt(lo16[:, 0]), cvt(hi16[:, 0]), cvt(lo16[:, 1])], 1)
    Ap, Bp, Cp, lo = r[:, 2].astype(np.float64), r[:, 3].astype(np.float64), r[:, 4].astype(np.float64), r[:, 5].astype(np.float64)
    return dict(u=r[:, 0], v=r[:, 1], A=-2 * LN2 * Ap, B=-LN2 * Bp, C=-2 * LN2 * Cp,
                opac=np.exp2(lo), rgb=rgb.astype(np.float64))


def rel_check(got: np.ndarray, ref: np.ndarray, rtol: float, what: str, floor: float = 1e-2):
    """Per column: entries with |ref| >= floor * max|ref| within rtol relative,
    every entry within rtol * max|ref| (max-norm relative)."""
    got = np.atleast_2d(np.asarray(got, np.float64).reshape(len(got), -1))
    ref = np.atleast_2d(np.asarray(ref, np.float64).reshape(len(ref), -1))
    for c in range(ref.shape[1]):
        r, g = ref[:, c], got[:, c]
        scale = np.max(np.abs(r)) if r.size else 0.0
        if scale == 0.0:
            assert np.max(np.abs(g)) <= 1e-12, f"{what}[{c}]: expected zeros"
            continue
        err = np.abs(g - r)
        assert err.max() <= rtol * scale, f"{what}[{c}]: max err {err.max():.3e} > {rtol} * {scale:.3e}"
        big = np.abs(r) >= floor * scale
        rel = err[big] / np.abs(r[big])
        assert rel.max() <= rtol, f"{what}[{c}]: rel err {rel.max():.3e} on significant entries"


def oracle_lists(cam, kp) -> tuple:
    """All tile lists of a view from the oracle: (vals, ranges)."""
    vals, ranges, off = [], np.zeros((cam.n_tiles, 2), np.int64), 0
    for t in range(cam.n_tiles):
        ids = O.tile_list(kp, t % cam.tiles_x, t // cam.tiles_x)
        ranges[t] = (off, off + len(ids))
        off += len(ids)
        vals.append(ids)
    return (np.concatenate(vals) if vals else np.zeros(0, np.uint32)), ranges


# ---------------------------------------------------------------------------
# 16-bit storage (SH coefficients and record colours in BF16 / FP16)
# ---------------------------------------------------------------------------

STORAGE_KIND = {1: "bf16", 2: "f16"}       # GS_BF16, GS_F16
# FP32 evaluation of a colour (16 SH terms, each with a few ulp of error)
# stays well inside this distance of the FP64 value
COLOUR_MARGIN = 8e-6
GROUPS = dict(means=(0, 3), log_scales=(3, 6), quats=(6, 10), logits=(10, 11), sh=(11, 59))


def _hash_level(c):
    """The 16-level quantisation of a colour channel (Sec. IV-C1): 8 bits as
    floor(c 255 + 0.5) clamped, then c8 >> 4."""
    return np.clip(np.floor(np.asarray(c, np.float64) * 255.0 + 0.5), 0, 255).astype(np.int64) >> 4


def storage_scene(scene, cams, dtype, margin=COLOUR_MARGIN, rounds=40, only=None, hash_safe=False):
    """A copy of `scene` prepared for parity of the 16-bit storage path
    (dtype GS_BF16 / GS_F16) or of colour hashing (hash_safe).

    The SH coefficients are rounded to the storage format (what the GPU
    reads).  The GPU evaluates each colour in FP32 and rounds it to the
    record's 16-bit format; the oracle evaluates it in FP64 and rounds it
    with O.round_storage.  The two agree unless the colour lies within FP32
    error of a point where that rounding changes (a midpoint between two
    16-bit values) or of the max(0, .) clamp; with hash_safe, also of a point
    where the colour's 16-level hash quantisation changes (FP32 records).
    While some visible (Gaussian, channel) of some view lies within `margin`
    of one, its DC coefficient is raised by 0.004 (then rounded), which moves
    the colour by at least 5.6e-4.  `only` (indices) limits the preparation
    to the Gaussians a comparison reads.  This prepares the input from the
    oracle's own colours only."""
    kind = STORAGE_KIND.get(dtype)
    sc = scene.subset(np.arange(scene.n))
    rnd = (lambda x: O.round_storage(x, kind)) if kind else (lambda x: x)
    sc.sh = rnd(sc.sh).astype(np.float32)
    idx = np.arange(sc.n) if only is None else np.asarray(only, np.int64)
    for _ in range(rounds):
        sub = sc.subset(idx)
        bad = np.zeros((sub.n, 3), bool)
        for cam in cams:
            kp = O.keypath(cam, sub)
            pr = O.project(cam, sub, kp)
            pre = pr["rgb_pre"]
            lo, hi = np.maximum(pre - margin, 0.0), np.maximum(pre + margin, 0.0)
            flip = np.abs(pre) < margin
            if kind:
                flip |= O.round_storage(lo, kind) != O.round_storage(hi, kind)
            if hash_safe:
                flip |= _hash_level(lo) != _hash_level(hi)
            bad |= flip & (kp["touched"] > 0)[:, None]
        if not bad.any():
            return sc
        i, ch = np.nonzero(bad)
        sc.sh[idx[i], 0, ch] = rnd(sc.sh[idx[i], 0, ch].astype(np.float64) + 0.004)
    raise AssertionError("colours still next to a rounding point after the nudges")


def storage_refs(sc, cams, dtype, window=None):
    """Oracle of the 16-bit storage path for each view: FP64 projection of
    the (already rounded) SH, the record colour rounded to the storage format,
    FP64 blending of that colour.  GS_F32: the plain FP64 oracle."""
    kind = STORAGE_KIND.get(dtype)
    refs = []
    for cam in cams:
        kp = O.keypath(cam, sc)
        pr = dict(O.project(cam, sc, kp))
        if kind:
            pr["rgb"] = O.round_storage(pr["rgb"], kind)
        refs.append(dict(kp=kp, proj=pr, r=O.render(cam, kp, pr, window)))
    return refs


def rel_errors(got, ref, floor: float = 1e-2):
    """(max error / max |ref|, median relative error over entries with
    |ref| >= floor max |ref|), pooled over the columns of one group."""
    got = np.asarray(got, np.float64).reshape(len(got), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    scale = np.abs(ref).max(axis=0, keepdims=True)
    scale = np.where(scale > 0, scale, 1.0)
    err = np.abs(got - ref)
    big = np.abs(ref) >= floor * scale
    rel = err[big] / np.abs(ref[big])
    return float((err / scale).max()), float(np.median(rel)) if rel.size else 0.0


def blending_at_flagged(cam, kp, proj, flag, margin=1e-3):
    """Gaussians that blend at some flagged pixel (alpha there at least
    (1 - margin)/255): the only ones whose gradient a decision flipped at
    that pixel can change.  A Gaussian gets gradient from a pixel only where
    it blends, and a flipped decision at a pixel changes the transmittance and
    the colour behind of exactly the Gaussians blending there."""
    out = np.zeros(kp["depth"].shape[0], bool)
    for y, x in np.argwhere(flag != 0):
        ids = O.tile_list(kp, x // 16, y // 16).astype(np.int64)
        if ids.size == 0:
            continue
        dx = x + 0.5 - proj["mean2d"][ids, 0]
        dy = y + 0.5 - proj["mean2d"][ids, 1]
        A, B, C = proj["conic"][ids, 0], proj["conic"][ids, 1], proj["conic"][ids, 2]
        alpha = np.minimum(0.99, proj["opac"][ids] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy))
        out[ids[alpha >= (1.0 - margin) / 255.0]] = True
    return out

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

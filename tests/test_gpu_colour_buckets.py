"""Colour hashing of tile lists (Sec. IV-C1) through the C ABI against the
oracle: bucket counts and distinct buckets per tile bit for bit (the
quantisation is FP32 with every operation rounded on both sides); colour and
opacity sums within 1e-4 relative (FP32 shared-memory atomics per tile, then
FP64 across tiles, in no fixed order; opacity through ex2.approx)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _synthetic(n, T, seed):
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(-0.1, 1.2, (n, 3)).astype(np.float32)
    rgb[: n // 10] = (rng.integers(0, 256, (n // 10, 3)) + 0.5).astype(np.float32) / np.float32(255.0)  # half-way
    lo = rng.uniform(-8.0, 0.0, n).astype(np.float32)
    lens = rng.integers(0, 200, T)
    lens[rng.random(T) < 0.1] = 0                                  # empty tiles
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    ranges = np.stack([starts, starts + lens], 1).astype(np.uint32)
    vals = rng.integers(0, n, int(lens.sum())).astype(np.uint32)
    return rgb, lo, ranges, vals


def _records(rgb, lo, dtype):
    n = len(lo)
    if dtype == L.GS_F32:
        rec = np.zeros((n, 12), np.float32)
        rec[:, 5], rec[:, 6], rec[:, 7], rec[:, 8] = lo, rgb[:, 0], rgb[:, 1], rgb[:, 2]
        return rec, rgb
    t = torch.bfloat16 if dtype == L.GS_BF16 else torch.float16
    h = torch.from_numpy(rgb).to(t)
    bits = h.view(torch.int16).numpy().astype(np.uint16).astype(np.uint32)
    rec = np.zeros((n, 8), np.float32)
    rec[:, 5] = lo
    rec.view(np.uint32)[:, 6] = bits[:, 0] | (bits[:, 1] << 16)
    rec.view(np.uint32)[:, 7] = bits[:, 2]
    return rec, h.float().numpy()


def _run(T, ranges, vals, rec, dtype):
    dev = "cuda"
    count = torch.zeros(4096, dtype=torch.int64, device=dev)
    sums = torch.zeros(4 * 4096, dtype=torch.float64, device=dev)
    distinct = torch.full((max(T, 1),), -1, dtype=torch.int32, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    L.gs_colour_buckets(T, t(ranges.view(np.int32)), t(vals.view(np.int32)), t(rec.ravel()), dtype, count, sums,
                        distinct)
    torch.cuda.synchronize()
    return count.cpu().numpy(), sums.cpu().numpy().reshape(4, 4096), distinct[:T].cpu().numpy()


@pytest.mark.parametrize("dtype", [L.GS_F32, L.GS_BF16, L.GS_F16])
def test_colour_buckets_match_oracle(dtype):
    rgb, lo, ranges, vals = _synthetic(50_000, 3001, seed=dtype)
    rec, rgb_seen = _records(rgb, lo, dtype)
    count, sums, distinct = _run(len(ranges), ranges, vals, rec, dtype)
    c_ref, s_ref, d_ref = O.colour_buckets(ranges, vals, rgb_seen, lo)
    assert np.array_equal(count, c_ref)
    assert np.array_equal(distinct, d_ref)
    assert np.allclose(sums, s_ref, rtol=1e-4, atol=1e-6)


def test_colour_buckets_on_rendered_lists():
    """Kept-prefix lists of a projected scene (16-bit records): every entry is
    counted once and each tile's distinct buckets are between 1 and its
    length (0 for an empty list)."""
    scene, cams = S.skewed_scene(200_000, 0), [S.front_camera(640, 480)]
    fr = P.Frame(cams, scene.n, rgb_dtype=L.GS_BF16, prefix=True)
    fr.project(P.param_views(P.to_device_params(scene), scene.n))
    fr.bin_sort()
    torch.cuda.synchronize()
    count, sums, distinct = _run(fr.T, fr.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2),
                                 fr.vals.cpu().numpy().view(np.uint32), fr.splats.cpu().numpy(), L.GS_BF16)
    rg = fr.ranges.cpu().numpy().reshape(-1, 2).astype(np.int64)
    lens = rg[:, 1] - rg[:, 0]
    assert count.sum() == lens.sum() == int(fr.n_inst.item())
    assert np.all(distinct <= np.minimum(lens, 4096)) and np.all((distinct > 0) == (lens > 0))
    assert np.all(sums[3] >= 0)


def test_no_tiles_and_bad_dtype():
    count = torch.zeros(4096, dtype=torch.int64, device="cuda")
    sums = torch.zeros(4 * 4096, dtype=torch.float64, device="cuda")
    d = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.gs_colour_buckets(0, None, None, None, L.GS_F32, count, sums, d)
    with pytest.raises(L.GsError):
        L.gs_colour_buckets(1, d, d, d, 7, count, sums, d)

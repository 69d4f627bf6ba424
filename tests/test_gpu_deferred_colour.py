"""Deferred colour (Sec. II-A colour of a splat, evaluated only where the
blend loops read it): a frame that projects without SH and colours the
records its kept lists reference -- listed by the placement of the prefix
binning, and after a repair the records of the rebuilt lists
(gs_colour_records, gs_colour_repaired) -- renders exactly what a frame that
colours every record at projection renders: the same record bytes for every
listed record, the same image, transmittance and processed counts, bit for
bit, on one view and on a batch of three, without history, with the
previous step's processed counts as limits, and with limits cut so short
that a repair rebuilds lists."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _cams(views_n):
    if views_n == 1:
        return [S.front_camera(320, 240)]
    return S.ring_cameras(3, [(320, 240), (256, 200), (300, 180)])


def _frames(cams, scene, rgb_dtype, sh_dtype):
    params = P.to_device_params(scene)
    views = dict(P.param_views(params, scene.n))
    if sh_dtype != L.GS_F32:
        views["sh"] = views["sh"].to(torch.bfloat16 if sh_dtype == L.GS_BF16 else torch.float16)
    frames = [P.Frame(cams, scene.n, rgb_dtype=rgb_dtype, sh_dtype=sh_dtype, prefix=True, defer_colour=d)
              for d in (True, False)]
    return frames, views


def _step(frames, views, short_limits=False):
    for fr in frames:
        if short_limits:
            fr.tile_nproc.fill_(1)                 # prefixes cut at 66 entries: tiles get repaired
        fr.project(views)
        fr.bin_sort()
        fr.render()
    torch.cuda.synchronize()


def _listed(fr):
    """The entries of every tile's list (the kept prefixes and any lists a
    repair rebuilt after them), tile by tile."""
    rg = fr.ranges.view(-1, 2).cpu().numpy().astype(np.int64)
    vals = fr.vals.cpu().numpy()
    return np.concatenate([vals[x:y] for x, y in rg if y > x] + [np.zeros(0, vals.dtype)])


def _check_equal(frames):
    """The same list per tile (a repair may place the rebuilt lists in
    another order: the forward lists the tiles to repair in the order it
    finds them), every listed record bit for bit, identical outputs; returns
    the listed records."""
    a, b = frames
    assert a.check_errors() == 0 and b.check_errors() == 0
    la, lb = _listed(a), _listed(b)
    assert la.size > 0 and np.array_equal(la, lb)
    rec = L.SPLAT_BYTES[a.rgb_dtype] // 4
    kept = torch.from_numpy(np.unique(la).astype(np.int64)).cuda()
    ra = a.splats.view(-1, rec)[kept].view(torch.int32)
    rb = b.splats.view(-1, rec)[kept].view(torch.int32)
    assert torch.equal(ra, rb)                     # every listed record, bit for bit
    assert torch.equal(a.img.view(torch.int32), b.img.view(torch.int32))
    assert torch.equal(a.T_final.view(torch.int32), b.T_final.view(torch.int32))
    assert torch.equal(a.n_proc, b.n_proc)
    return kept


@pytest.mark.parametrize("views_n,rgb_dtype,sh_dtype", [(1, L.GS_BF16, L.GS_F32), (1, L.GS_F32, L.GS_BF16),
                                                         (3, L.GS_F16, L.GS_F32)])
def test_deferred_colour_renders_the_same(views_n, rgb_dtype, sh_dtype):
    scene = S.skewed_scene(200_000, 5)            # dense enough that many records lie behind every kept prefix
    cams = _cams(views_n)
    frames, views = _frames(cams, scene, rgb_dtype, sh_dtype)
    _step(frames, views)                           # no history: the coverage bound cuts the lists
    _check_equal(frames)
    _step(frames, views)                           # the previous step's processed counts as limits
    kept = _check_equal(frames)
    a = frames[0]
    VN = len(cams) * scene.n
    assert kept.numel() < VN                       # only some records are coloured
    # the placement listed each record once, only records the lists reference,
    # and every referenced record was marked (coloured) in this step
    listed = a.colour_list[:int(a.colour_count.item())].long()
    assert torch.unique(listed).numel() == listed.numel() and bool(torch.isin(listed, kept).all())
    assert bool((a.colour_mark[kept] == a.colour_epoch).all())
    if int(a.flag_count.item()) == 0:
        assert listed.numel() == kept.numel()
    # records no list references keep the zero colour the projection wrote
    rec = L.SPLAT_BYTES[a.rgb_dtype] // 4
    unused = torch.ones(VN, dtype=torch.bool, device="cuda")
    unused[kept] = False
    vis = (a.touched[:VN] > 0) & unused
    assert bool(vis.any())
    words = a.splats.view(-1, rec)[:VN][vis]
    colour = words[:, 6:9] if a.rgb_dtype == L.GS_F32 else words[:, 6:8]
    assert int((colour != 0).sum()) == 0


@pytest.mark.parametrize("views_n", [1, 3])
def test_deferred_colour_covers_repaired_lists(views_n):
    scene = S.skewed_scene(60_000, 6)
    cams = _cams(views_n)
    frames, views = _frames(cams, scene, L.GS_BF16, L.GS_F32)
    _step(frames, views)
    _step(frames, views, short_limits=True)
    flagged = int(frames[0].flag_count.item())
    assert flagged > 0                             # some tiles were repaired and re-rendered
    assert flagged == int(frames[1].flag_count.item())
    kept = _check_equal(frames)
    a = frames[0]
    assert kept.numel() > int(a.colour_count.item())   # records only the rebuilt lists reference
    assert bool((a.colour_mark[kept] == a.colour_epoch).all())


def test_colour_entries_refuse_bad_arguments():
    cam = S.front_camera(64, 64)
    fr = P.Frame([cam], 8, prefix=True)
    x = torch.zeros(64, device="cuda")
    with pytest.raises(L.GsError):                 # no SH
        L.gs_colour_records([cam], 8, x, None, L.GS_F32, fr.colour_list, fr.colour_count, fr.splats, L.GS_F32)
    with pytest.raises(L.GsError):                 # no tile ranges
        L.gs_colour_repaired([cam], 8, x, x, L.GS_F32, fr.vals, 16, fr.flag_tiles, fr.flag_count, None,
                             fr.colour_mark, 1, fr.splats, L.GS_F32)

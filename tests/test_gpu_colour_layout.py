"""Colour-layout ablation of the forward pass (Sec. V): planar or interleaved
colour, read in the blend loop or batch-loaded into shared memory.  The
layout changes where a colour is read from, never a value or the order of
the arithmetic, so every layout must give the production forward's image,
transmittance and processed counts bit for bit, and the oracle's image
within the image tolerance on unflagged pixels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2510_14564_gb300 import _lib as L
from paper_2510_14564_gb300 import pipeline as P
from paper_2510_14564_gb300 import scenes as S
from tests._util import IMG_ATOL

pytestmark = pytest.mark.gpu

CASES = {
    "uniform-10k-256x256": lambda: (S.uniform_scene(10_000, 0), [S.front_camera(256, 256)]),
    "ragged-250x190": lambda: (S.uniform_scene(6_000, 5), [S.front_camera(250, 190)]),
    "skewed-60k-3views": lambda: (S.skewed_scene(60_000, 3),
                                  S.ring_cameras(3, [(320, 240), (200, 300), (256, 256)])),
}


def _layouts(fr):
    VN = fr.V * fr.N
    planar = torch.empty(3 * VN, dtype=torch.float32, device="cuda")
    inter = torch.empty(3 * VN, dtype=torch.float32, device="cuda")
    L.gs_colour_arrays(VN, fr.splats, planar, inter)
    out = {}
    for name, layout in L.COLOUR_LAYOUTS.items():
        img = torch.full_like(fr.img, -1.0)
        T = torch.full_like(fr.T_final, -1.0)
        npx = torch.full_like(fr.n_proc, -1)
        colour = planar if "planar" in name else inter
        L.gs_render_fwd_colour(fr.cams, fr.N, fr.ranges, fr.vals, fr.splats, layout, colour, img, T, npx)
        out[name] = (img, T, npx)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prefix", [False, True])
@pytest.mark.parametrize("name", list(CASES))
def test_every_layout_gives_the_production_image(name, prefix):
    scene, cams = CASES[name]()
    params = P.to_device_params(scene)
    views = P.param_views(params, scene.n)
    fr = P.Frame(cams, scene.n, rgb_dtype=L.GS_F32, prefix=prefix)
    fr.project(views)
    fr.bin_sort()                 # kept prefixes without history: the guaranteed bound, nothing flagged
    fr.render()
    torch.cuda.synchronize()
    assert fr.check_errors() == 0
    if prefix:
        assert int(fr.flag_count.item()) == 0
    for layout, (img, T, npx) in _layouts(fr).items():
        assert torch.equal(img, fr.img), layout
        assert torch.equal(T, fr.T_final), layout
        assert torch.equal(npx, fr.n_proc), layout


def test_staged_interleaved_layout_matches_the_oracle():
    scene, cams = S.uniform_scene(10_000, 0), [S.front_camera(256, 256)]
    params = P.to_device_params(scene)
    fr = P.Frame(cams, scene.n, rgb_dtype=L.GS_F32)
    fr.project(P.param_views(params, scene.n))
    fr.bin_sort()
    img, T, npx = _layouts(fr)["interleaved_staged"]
    r = O.forward(cams[0], scene)
    ok = r["flag"] == 0
    assert ok.mean() > 0.98
    got = img.view(3, 256, 256).cpu().numpy()
    assert np.abs(got - r["img"])[:, ok].max() <= IMG_ATOL
    assert np.array_equal(npx.view(256, 256).cpu().numpy()[ok], r["n_proc"][ok])


def test_bad_layout_is_refused():
    scene, cams = S.uniform_scene(500, 1), [S.front_camera(64, 48)]
    fr = P.Frame(cams, scene.n, rgb_dtype=L.GS_F32)
    fr.project(P.param_views(P.to_device_params(scene), scene.n))
    fr.bin_sort()
    col = torch.zeros(3 * scene.n, device="cuda")
    with pytest.raises(L.GsError):
        L.gs_render_fwd_colour(fr.cams, fr.N, fr.ranges, fr.vals, fr.splats, 4, col, fr.img, fr.T_final,
                               fr.n_proc)

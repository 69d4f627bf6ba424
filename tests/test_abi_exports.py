"""The C-ABI library loads and exports every entry point include/gs103.h
declares (CPU only: no compute call is made)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "gs103.h"


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    names = re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2510_14564_gb300 import build as B
    return B.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_project_bwd",
              "gs_adam_step", "gs_l1_loss", "gs_tile_features", "gs_mlp_predict",
              "gs_mlp_train_step", "gs_sched_order"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(str(lib_path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    from paper_2510_14564_gb300 import _lib as L
    assert sorted(L.EXPORTS) == declared_functions()
    for n in L.EXPORTS:
        assert callable(getattr(L, n)), n


def test_host_only_calls(lib_path):
    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import scenes as S
    assert L.gs_version() >= 1
    assert L.lib().gs_strerror(L.GS_ERR_ARG).decode().startswith("invalid")
    cam = S.front_camera(1600, 1060)
    n = L.gs_bin_sort_workspace([cam], 1000, 50_000)
    assert n > 50_000 * 12
    assert L.gs_sched_order_workspace(6700) > 6700 * 16
    with pytest.raises(L.GsError):
        L.gs_bin_sort_workspace([cam], -1, 10)


def test_host_checks_of_the_later_entry_points(lib_path):
    """Argument checks that return before any device work (raw calls: the
    binding's wrappers ask torch for the current stream)."""
    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import scenes as S
    lib = L.lib()
    assert L.gs_densify_workspace(1000) > 4 * 1000 * 6
    assert L.gs_density_workspace(1000) > 4 * (1 << 24)          # the cell table
    with pytest.raises(L.GsError):
        L.gs_density_workspace(-1)
    z = [None] * 4
    assert lib.gs_density_stats(10, None, 0.0, 3, *z, None, None, None, 0, None) == L.GS_ERR_ARG   # r > 0
    assert lib.gs_density_stats(10, None, 0.1, 9, *z, None, None, None, 0, None) == L.GS_ERR_ARG   # k <= 8
    assert lib.gs_density_stats(10, None, 0.1, 3, *z, None, None, None, 0, None) == L.GS_ERR_ARG   # null buffers
    assert lib.gs_colour_buckets(1, None, None, None, 7, None, None, None, None) == L.GS_ERR_ARG   # record type
    assert lib.gs_colour_buckets(0, None, None, None, 0, None, None, None, None) == L.GS_OK        # no tiles
    cams = L.camera_array([S.front_camera(64, 48)])
    assert lib.gs_render_fwd_colour(cams, 1, 10, None, None, None, 0, None, None, None, None, None) == L.GS_ERR_ARG
    assert lib.gs_densify(-1, None, None, None, None, 0.0, 0, 0, None, None, None, None, 1, None, None, 0,
                          None, None) == L.GS_ERR_ARG
    assert lib.gs_densify(10, None, None, None, None, 0.0, 0, 100, None, None, None, None, 9, None, None, 0,
                          None, None) == L.GS_ERR_ARG                # null output count / bad shadow type

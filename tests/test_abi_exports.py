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

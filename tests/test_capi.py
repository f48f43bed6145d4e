"""The C ABI library builds, loads without a GPU and exports every entry
point that include/gs.h declares (no compute calls)."""
import ctypes
import os
import re

from paper_2509_05216_gb300 import build as gsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_path():
    names = declared_functions()
    for f in ["gs_project", "gs_bin_sort", "gs_raster_fwd", "gs_raster_bwd", "gs_adam", "gs_create",
              "gs_destroy", "gs_sync"]:
        assert f in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gsbuild.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_the_exports():
    from paper_2509_05216_gb300 import gs
    assert set(gs.EXPORTS) <= set(declared_functions())

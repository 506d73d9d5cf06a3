"""The C ABI library builds, loads without a GPU and exports every symbol
include/gdist.h declares; the binding covers the same names."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gdist.h")).read()
    return sorted(set(re.findall(r"GD_API\s+[\w\s\*]+?\b(gd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_11244_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gd_ctx_create", "gd_mesh_create", "gd_bvh_build", "gd_min_distance", "gd_max_distance",
              "gd_batch_query", "gd_serve_submit", "gd_serve_poll", "gd_mesh_destroy", "gd_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2411_11244_gb300 import gdist
    assert sorted(gdist.EXPORTS) == _declared()
    for n in _declared():
        assert callable(getattr(gdist, n)), n


def test_no_device_fails_loudly(lib):
    """Without a CUDA device the engine refuses instead of computing on the CPU."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2411_11244_gb300 import gdist
    with pytest.raises(gdist.GdError):
        gdist.gd_ctx_create(0)


def test_struct_layouts():
    from paper_2411_11244_gb300 import gdist
    assert ctypes.sizeof(gdist.gd_result) == 80
    assert ctypes.sizeof(gdist.gd_query) == 8 + 8 + 96 + 96 + 8 + 8

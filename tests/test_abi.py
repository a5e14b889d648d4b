"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/eb.h declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "eb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eb_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2604_11959_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("eb_geom_build", "eb_flux_div", "eb_wsrd", "eb_step"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_version_and_error_string(lib):
    lib.eb_version.restype = ctypes.c_int
    lib.eb_last_error.restype = ctypes.c_char_p
    assert lib.eb_version() >= 100
    assert isinstance(lib.eb_last_error(), bytes)


def test_binding_names_match(lib):
    from paper_2604_11959_gb300 import eb
    assert sorted(eb.EXPORTED_SYMBOLS) == declared_symbols()

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


def _header_struct_fields(name):
    """(field, count) of a typedef struct in include/eb.h, in order."""
    src = open(os.path.join(ROOT, "include", "eb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"([A-Za-z_][A-Za-z0-9_ ]*?)\s+(.+)$", decl)
        for var in m.group(2).split(","):
            var = var.strip().lstrip("*").strip()
            vm = re.match(r"(\w+)(?:\[(\d+)\])?$", var)
            out.append((vm.group(1), int(vm.group(2) or 1)))
    return out


def test_info_struct_binding_matches_the_header():
    """The Python mirror of eb_geom_info_t has the header's fields in the
    header's order, with the same array lengths (an out-of-order field would
    shift every later one)."""
    from paper_2604_11959_gb300 import eb
    want = _header_struct_fields("eb_geom_info_t")
    got = []
    for fname, ftype in eb.GeomInfo._fields_:
        got.append((fname, getattr(ftype, "_length_", 1)))
    assert got == want


def test_desc_and_state_bindings_match_the_header():
    from paper_2604_11959_gb300 import eb
    assert [(n, 1) for n, _ in eb._Desc._fields_] == _header_struct_fields("eb_desc")
    assert [(n, 1) for n, _ in eb._State._fields_] == _header_struct_fields("eb_state")

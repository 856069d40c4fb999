"""The C-ABI library builds, loads and exports every entry point include/gs.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgs():
    from paper_2603_09632_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(gs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for need in ("gs_project", "gs_bin_tiles", "gs_render_fwd", "gs_render_bwd",
                 "gs_workspace_create", "gs_workspace_destroy", "gs_status_string"):
        assert need in names


def test_every_status_returning_call_documents_its_errors():
    # each gs_status function's comment states its error behaviour ("Errors: ...", "Errors
    # as <other call>" or the GS_ERR_ codes it returns), and the four hot-path calls cite
    # the passage of the paper they compute
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    decls = list(re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*gs_status\s+(gs_\w+)\s*\(", src, re.S))
    assert len(decls) >= 20
    for m in decls:
        doc, name = m.group(1), m.group(2)
        assert "Errors" in doc or "GS_ERR_" in doc, name
        if name in ("gs_project", "gs_bin_tiles", "gs_render_fwd", "gs_render_bwd"):
            assert re.search(r"Eq\. \d|App\. [A-E]|Sec\. \d", doc), name


def test_every_declared_symbol_is_exported(libgs):
    missing = [n for n in declared_functions() if not hasattr(libgs, n)]
    assert not missing, missing


def test_status_strings(libgs):
    libgs.gs_status_string.restype = ctypes.c_char_p
    libgs.gs_status_string.argtypes = [ctypes.c_int]
    assert libgs.gs_status_string(0) == b"ok"
    assert libgs.gs_status_string(4) == b"device-side error"
    assert libgs.gs_status_string(999) == b"unknown status"


def test_null_arguments_rejected(libgs):
    libgs.gs_project.argtypes = [ctypes.c_void_p] * 4
    libgs.gs_bin_tiles.argtypes = [ctypes.c_void_p] * 3
    libgs.gs_workspace_create.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert libgs.gs_project(None, None, None, None) == 1          # GS_ERR_ARG
    assert libgs.gs_bin_tiles(None, None, None) == 1
    assert libgs.gs_workspace_create(None, 0) == 1
    libgs.gs_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert libgs.gs_workspace_bytes(None, None) == 1


def test_binding_names_match_header():
    src = open(os.path.join(ROOT, "paper_2603_09632_gb300", "_lib.py")).read()
    for n in ("gs_project", "gs_bin_tiles", "gs_render_fwd", "gs_render_bwd"):
        assert f"def {n}(" in src

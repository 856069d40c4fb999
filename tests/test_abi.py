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


def _header_signatures():
    """name -> (return kind, [parameter kinds]) of every function gs.h declares."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "gs.h")).read(), flags=re.S)
    out = {}
    for ret, name, args in re.findall(r"\b(gs_status|void|int64_t|const char\s*\*)\s+(gs_\w+)\s*\(([^)]*)\)\s*;", src):
        params = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        out[name] = (_c_kind(ret), [_c_kind(p) for p in params])
    return out


def _c_kind(decl):
    """Kind of a C type (as it crosses the ABI): pointer, i32, i64, u64, f32 or none."""
    d = " ".join(decl.split())
    if "*" in d:
        return "ptr"
    t = d.rsplit(" ", 1)[0] if " " in d else d
    t = t.replace("const ", "")
    if t in ("void",):
        return "none"
    if t in ("int", "int32_t", "gs_status"):
        return "i32"
    return {"int64_t": "i64", "uint64_t": "u64", "float": "f32", "double": "f64"}[t]


def _binding_signatures():
    """name -> (return kind, [argument kinds]) of the ctypes declarations in _lib.py, read
    from its source (the signature table of its loader) without loading the library."""
    import ast
    src = open(os.path.join(ROOT, "paper_2603_09632_gb300", "_lib.py")).read()
    table = None
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Assign) and any(getattr(t, "id", None) == "sig" for t in node.targets):
            table = node.value
    assert isinstance(table, ast.Dict)

    class _C:   # the ctypes names the table uses, mapped to ABI kinds
        c_void_p = c_char_p = "ptr"
        c_int = c_int32 = "i32"
        c_int64 = "i64"
        c_uint64 = "u64"
        c_float = "f32"
        c_double = "f64"

        @staticmethod
        def POINTER(_):
            return "ptr"

    env = {"C": _C, "P": "ptr", "i64": "i64", "i32": "i32", "st": "i32", "None": None}
    out = {}
    for k, v in zip(table.keys, table.values):
        args, res = eval(compile(ast.Expression(v), "<sig>", "eval"), env)
        out[k.value] = ("none" if res is None else res, list(args))
    return out


def test_binding_signatures_match_header():
    # every function of gs.h has a ctypes declaration with the same number and kinds of
    # arguments (pointer, 32- or 64-bit integer, float, double) and the same return kind
    hdr, bind = _header_signatures(), _binding_signatures()
    assert set(hdr) == set(bind), (sorted(set(hdr) - set(bind)), sorted(set(bind) - set(hdr)))
    bad = {n: (hdr[n], bind[n]) for n in hdr if hdr[n] != bind[n]}
    assert not bad, bad

"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/stokes_mg.h (no compute calls: no GPU needed)."""
import os
import re

import pytest

from paper_1911_05888_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "stokes_mg.h")).read()
    return set(re.findall(r"^\s*(?:int|const char\*)\s+(stk_\w+)\s*\(", src, re.M))


@pytest.fixture(scope="module")
def lib_path():
    return build.build()


def test_header_and_binding_agree():
    assert declared_symbols() == set(native.SIGNATURES)


def test_library_exports_every_symbol(lib_path):
    assert native.exported_symbols(lib_path) == declared_symbols()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1911_05888_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def _declarations():
    """name -> list of C parameter types, parsed from the header."""
    src = open(os.path.join(ROOT, "include", "stokes_mg.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    out = {}
    for m in re.finditer(r"(?:int|const char\*)\s+(stk_\w+)\s*\(([^)]*)\)\s*;", src):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = [re.sub(r"\s+\w+$", "", p) if not p.endswith("*") else p for p in params]
    return out


def _category_c(t):
    t = t.replace("const ", "").strip()
    if "*" in t:
        return "ptr"
    return {"int": "i32", "int64_t": "i64", "uint64_t": "u64", "double": "f64", "float": "f32", "size_t": "u64"}[t]


def _category_ctypes(a):
    import ctypes
    if a in (ctypes.c_void_p,) or (isinstance(a, type) and issubclass(a, ctypes._Pointer)):
        return "ptr"
    if isinstance(a, type) and issubclass(a, ctypes.Array):
        return "ptr"
    return {ctypes.c_int: "i32", ctypes.c_int64: "i64", ctypes.c_uint64: "u64", ctypes.c_double: "f64",
            ctypes.c_float: "f32", ctypes.c_size_t: "u64"}.get(a, "ptr" if a is ctypes.c_char_p else repr(a))


def test_binding_argument_types_match_header():
    """Every ctypes signature has the header's arity, and each argument is of
    the same kind (pointer, 32/64-bit integer, double, float)."""
    decl = _declarations()
    assert set(decl) == set(native.SIGNATURES)
    for name, cparams in decl.items():
        py = native.SIGNATURES[name]
        assert len(py) == len(cparams), (name, cparams, py)
        for k, (ct, pt) in enumerate(zip(cparams, py)):
            assert _category_c(ct) == _category_ctypes(pt), (name, k, ct, pt)

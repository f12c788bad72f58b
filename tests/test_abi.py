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

"""The C-ABI library builds, loads and exports every entry point that
include/cd_api.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cd_api.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:cd_status|void|const char\s*\*)\s*(cd_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cd_create_system", "cd_detect_contacts", "cd_solve_contacts", "cd_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1104_3516_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1104_3516_gb300 import cd
    bound = {name for name, _, _ in cd.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_oracle_is_not_reachable_from_the_product_package():
    pkg = os.path.join(ROOT, "paper_1104_3516_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".c", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "cd_oracle" not in text, f

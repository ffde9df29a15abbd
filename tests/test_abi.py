"""The C-ABI library builds for sm_103a, loads, and exports every function include/mpk.h declares."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "mpk.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mpk_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    import paper_2405_12525_gb300 as mpk
    return mpk.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mpk_build_levels", "mpk_plan", "mpk_apply", "mpk_cheb_filter"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(mpk_[a-z0-9_]+)\b", out))
    missing = [f for f in _declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_loads_and_lists_all_symbols(lib_path):
    import paper_2405_12525_gb300 as mpk
    lib = mpk.load()
    for f in _declared_functions():
        assert hasattr(lib, f), f
    assert sorted(mpk.EXPORTED_SYMBOLS) == _declared_functions()


def test_status_strings_without_gpu(lib_path):
    import paper_2405_12525_gb300 as mpk
    lib = mpk.load()
    assert lib.mpk_status_string(0) == b"ok"
    assert lib.mpk_status_string(4) == b"device wait timed out"

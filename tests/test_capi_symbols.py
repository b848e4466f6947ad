"""The C-ABI library builds, loads and exports every entry point its header declares.

Runs without a GPU: only host-side calls (status strings, version, argument
checks that fail before any device work) are made.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bg_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2505_22675_gb300 import build
    build.build()
    from paper_2505_22675_gb300 import _capi
    return _capi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"bg_ctx_create", "bg_grid_create", "bg_soundings_upload", "bg_interp_idw",
            "bg_interp_okrige"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings_and_version(lib):
    import paper_2505_22675_gb300 as bg
    assert lib.bg_status_str(0) == b"BG_OK"
    assert lib.bg_status_str(-2) == b"BG_ERR_OOM_BUDGET"
    assert lib.bg_status_str(-4) == b"BG_ERR_TIMEOUT"
    assert "sm_103a" in bg.version()


def test_null_arguments_are_rejected_without_device_work(lib):
    assert lib.bg_grid_create(None, 0, 0, 2, 1, 1, None) == -1
    assert lib.bg_soundings_destroy(None) == -1
    assert lib.bg_interp_idw(None, None, 8, ctypes.c_float(2.0), None, None, None) == -1
    assert b"NULL" in lib.bg_last_error()


def test_oracle_and_library_share_no_source():
    """The oracle and the CUDA path are independent: no file includes or imports the other."""
    csrc = os.path.join(ROOT, "paper_2505_22675_gb300")
    for dirpath, _, files in os.walk(csrc):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+\"?(\w+)", text), fn
    text = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "bathygrid" not in text and "paper_2505_22675_gb300" not in text

"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        text = re.sub(r"typedef[^;]*;", " ", text)
        for m in re.finditer(r"\b(cb_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cb_spgemm", "cb_spgemm_ex", "cb_csr_free", "cb_ctx_create", "cb_ctx_destroy",
                 "cb_status_str", "cb_last_error", "cb_row_stats", "cb_row_nnz",
                 "cb_exclusive_scan"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2106_14402_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2106_14402_gb300 import cb
    assert set(declared_functions()) <= set(cb.exported_symbols())


def test_status_strings_without_gpu():
    from paper_2106_14402_gb300 import cb
    lib = cb.load()
    assert lib.cb_status_str(0) == b"ok"
    assert b"too small" in lib.cb_status_str(9)


def test_debug_library_exports_the_same_symbols():
    from paper_2106_14402_gb300 import build
    path = build.build(check=True)
    assert path.endswith("libcb_check.so")
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing

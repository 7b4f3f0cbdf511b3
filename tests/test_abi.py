"""The C-ABI library builds, loads and exports every symbol its header
declares.  No compute call: this runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nnsemd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("nnsemd_create", "nnsemd_destroy", "nnsemd_solve", "nnsemd_solve_batched",
                 "nnsemd_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2401_07378_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.nnsemd_abi_version.restype = ctypes.c_int
    assert lib.nnsemd_abi_version() == 4
    lib.nnsemd_status_string.restype = ctypes.c_char_p
    assert lib.nnsemd_status_string(0) == b"NNSEMD_OK"
    assert lib.nnsemd_status_string(9) == b"NNSEMD_ERR_CAPACITY"


def test_binding_loads_and_matches_struct_sizes():
    from paper_2401_07378_gb300 import nnsemd
    assert ctypes.sizeof(nnsemd.nnsemd_options) == 40
    assert ctypes.sizeof(nnsemd.nnsemd_plan) == 40
    assert ctypes.sizeof(nnsemd.nnsemd_stats) == 96
    assert nnsemd.nnsemd_stats.near_ties.offset == 80
    assert nnsemd.nnsemd_stats.widened.offset == 88
    assert ctypes.sizeof(nnsemd.nnsemd_config) == 24
    assert nnsemd.abi_version() == 4


def test_null_context_is_rejected_without_a_gpu():
    from paper_2401_07378_gb300 import nnsemd
    lib = nnsemd._lib
    assert lib.nnsemd_destroy(None) == 0
    assert lib.nnsemd_set_stream(None, None) == 1
    assert lib.nnsemd_solve(None, None, None, 0, None, None, 0, 0, None, None, None, None) == 1
    out = ctypes.c_void_p()
    assert lib.nnsemd_create(None, None) == 1

"""The C-ABI library loads and exports every entry point include/psht.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "psht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psht_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("psht_plan_create", "psht_plan_synthesis", "psht_plan_adjoint", "psht_plan_destroy",
                 "psht_synthesis", "psht_adjoint_synthesis", "psht_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2603_17166_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.psht_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.psht_version()


def test_estimate_bytes_without_gpu():
    from paper_2603_17166_gb300 import estimate_bytes

    b = estimate_bytes(2, 4096, 0.6059, 20_000_000, 1e-10, "fp64")
    assert 1e9 < b < 2e10
    assert estimate_bytes(2, 4096, 0.6059, 20_000_000, 1e-5, "fp32") < b

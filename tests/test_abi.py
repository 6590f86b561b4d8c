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


def test_rotation_entry_points_validate_on_the_host():
    """Arguments are checked before any device work, so these run without a GPU."""
    from paper_2603_17166_gb300 import psht

    L = psht.lib()
    P = ctypes.c_void_p
    h = P()
    assert L.psht_rotator_create(-1, 2, None, ctypes.byref(h)) == -22
    assert L.psht_rotator_create(70000, 2, None, ctypes.byref(h)) == -22
    assert b"lmax" in L.psht_last_error()
    assert L.psht_rotator_create(10, 2, None, None) == -22
    # bytes: coefficient table + two intermediate sets (complex) + log-factorials + phase tables
    n = 4097 * 4098 // 2
    assert L.psht_rotator_bytes(4096, 2) == n * 8 * 3 + (2 * 4096 + 2) * 8 + 3 * 4097 * 8
    assert L.psht_rotator_bytes(4096, 1) == n * 16 * 3 + (2 * 4096 + 2) * 8 + 3 * 4097 * 16
    assert L.psht_patch_rotation(None, None, 0, None, None, None) == -22
    assert L.psht_rotate_points(0.0, 0.0, 0.0, None, None, -1, None, None, None, None) == -22
    # a patch-frame plan holds a rotator, the rotated a_lm and, for spin > 0, two per-point arrays
    b0 = L.psht_estimate_bytes(2, 1024, 0.6, 1_000_000, 1e-5, 2)
    b1 = L.psht_estimate_bytes(2, 1024, 0.6, 1_000_000, 1e-5, 2 | 8)
    assert b1 - b0 == L.psht_rotator_bytes(1024, 2) + 2 * (1025 * 1026 // 2) * 8 + 2 * 1_000_000 * 8
    assert L.psht_plan_create(2, 64, None, None, 0, 1e-5, 16, None, ctypes.byref(h)) == -22  # unknown flag

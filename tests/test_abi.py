"""The C ABI library loads and exports every function include/tnsk.h declares
(no GPU calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "tnsk.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:tnsk_status|const char\*)\s+(tnsk_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("tnsk_create", "tnsk_destroy", "tnsk_estimate", "tnsk_estimate_batch", "tnsk_m1_sketch",
                 "tnsk_count_sketch", "tnsk_sync", "tnsk_status_string", "tnsk_last_error"):
        assert want in names


def test_library_builds_and_exports_every_symbol():
    import ctypes
    import shutil

    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    from paper_2603_07387_gb300 import build, tnsk

    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(tnsk.SYMBOLS)
    # status strings need no device
    lib.tnsk_status_string.restype = ctypes.c_char_p
    assert lib.tnsk_status_string(-2) == b"TNSK_ERR_CYCLIC"

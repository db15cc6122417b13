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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of tnsk_tensor, tnsk_rung, tnsk_network and tnsk_params have
    the C layout (sizes and field offsets from a program compiled against the header)."""
    import ctypes
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    from paper_2603_07387_gb300 import tnsk

    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "tnsk.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu\\n", sizeof(tnsk_tensor), offsetof(tnsk_tensor, dtype), '
        "offsetof(tnsk_tensor, rung), sizeof(tnsk_rung));\n"
        '  printf("%zu %zu %zu\\n", offsetof(tnsk_rung, d), sizeof(tnsk_network), sizeof(tnsk_params));\n'
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(tnsk._Tensor), tnsk._Tensor.dtype.offset, tnsk._Tensor.rung.offset,
            ctypes.sizeof(tnsk._Rung), tnsk._Rung.d.offset, ctypes.sizeof(tnsk._Network),
            ctypes.sizeof(tnsk._Params)]
    assert got == want


def test_rung_factors_are_checked_on_the_host():
    torch = pytest.importorskip("torch")
    from paper_2603_07387_gb300 import tnsk

    r = tnsk.Rung(torch.zeros(3, 4, 5), torch.zeros(6, 4, 7))
    assert r.shape == (18, 35) and r.dim() == 2 and r.numel() == 18 * 35
    with pytest.raises(ValueError):
        tnsk.Rung(torch.zeros(3, 4, 5), torch.zeros(6, 2, 7))  # unequal shared dims
    with pytest.raises(ValueError):
        tnsk.Rung(torch.zeros(3, 4), torch.zeros(6, 4, 7))


def test_binding_kernel_kinds_follow_the_header():
    """tnsk_profile_read fills one slot per tnsk_kernel_kind: the binding's names are in
    the header's order and as many as TNSK_KERNEL_KINDS."""
    from paper_2603_07387_gb300 import tnsk

    with open(os.path.join(ROOT, "include", "tnsk.h")) as f:
        src = f.read()
    kinds = {int(v): k for k, v in re.findall(r"TNSK_K_(\w+)\s*=\s*(\d+)", src)}
    total = int(re.search(r"TNSK_KERNEL_KINDS\s*=\s*(\d+)", src).group(1))
    assert sorted(kinds) == list(range(total))
    assert len(tnsk.KERNEL_KINDS) == total
    assert [kinds[i].lower() for i in range(total)] == list(tnsk.KERNEL_KINDS)

"""The C-ABI library builds, loads and exports every function that
include/frobinv.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "frobinv.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_01239_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for required in ("frob_inv", "frob_inv_hpd", "cplx_lu_inv", "cplx_chol_inv", "frob_workspace_bytes",
                     "frob_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"libfrobinv.so does not export {name}"


def test_host_only_calls(lib):
    """Calls that touch no device: sizes, status strings, argument checks."""
    lib.frob_workspace_bytes.restype = ctypes.c_size_t
    lib.frob_workspace_bytes.argtypes = [ctypes.c_int] * 4
    assert lib.frob_workspace_bytes(0, 256, 1, 0) > 5 * 256 * 256 * 8
    assert lib.frob_workspace_bytes(0, 0, 1, 0) == 0
    assert lib.frob_workspace_bytes(9, 16, 1, 0) == 0
    # fp32 planes are half the size of fp64 planes
    assert lib.frob_workspace_bytes(1, 512, 4, 1) < lib.frob_workspace_bytes(1, 512, 4, 0)
    lib.frob_status_str.restype = ctypes.c_char_p
    assert lib.frob_status_str(2) == b"FROB_ERR_SINGULAR"
    # argument errors return synchronously, before any launch
    lib.frob_inv.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.frob_inv.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_int64,
                             ctypes.c_int64, vp, vp, ctypes.c_size_t, vp, vp]
    assert lib.frob_inv(0, 1, 16, 1, 1, 4096, 1, 1, None, 256, 1 << 20, 512, None) == 1      # n < 1
    assert lib.frob_inv(4, 1, 16, 3, 16, 4096, 4, 16, None, 256, 1 << 20, 512, None) == 1     # ldm < n
    assert lib.frob_inv(4, 1, None, 4, 16, 4096, 4, 16, None, 256, 1 << 20, 512, None) == 1   # NULL input
    assert lib.frob_inv(4, 1, 4096, 4, 16, 4096, 4, 16, None, 256, 1 << 20, 512, None) == 1   # in == out
    assert lib.frob_inv(4, 1, 16, 4, 16, 4096, 4, 16, None, 256, 8, 512, None) == 7          # ws too small
    assert lib.frob_inv(4, 1, 16, 4, 16, 4096, 4, 16, None, 257, 1 << 20, 512, None) == 7    # misaligned ws

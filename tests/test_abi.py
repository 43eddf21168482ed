"""The C-ABI library loads and exports every entry point include/*.h declares; host-side
argument checks answer without touching the GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text,
                              flags=re.M):
            names.append(mt.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1210_0800_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIBRARY)


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("ls_solve_dd", "ls_solve_qd", "mgs_qr_dd", "mgs_qr_qd", "mgs_workspace_bytes"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_argument_checks(lib):
    """Bad arguments are rejected on the host before any CUDA call."""
    from paper_1210_0800_gb300 import _binding

    L = _binding.load()
    vp = ctypes.c_void_p
    good = vp(4096)
    st = vp(8192)
    # null A
    assert L.ls_solve_dd(None, 4, good, good, None, 0, None, 4, 4, good, 1 << 20, st, None) == 1
    # m < n
    assert L.ls_solve_dd(good, 4, good, good, None, 0, None, 3, 4, good, 1 << 20, st, None) == 1
    # lda < m
    assert L.ls_solve_qd(good, 3, good, good, None, 0, None, 4, 4, good, 1 << 20, st, None) == 1
    # misaligned A
    assert L.mgs_qr_dd(vp(4100), 4, good, 4, 4, 4, good, 1 << 20, st, None) == 1
    # n < 1
    assert L.mgs_qr_qd(good, 4, good, 4, 4, 0, good, 1 << 20, st, None) == 1
    # QR needs R
    assert L.mgs_qr_dd(good, 4, None, 4, 4, 4, good, 1 << 20, st, None) == 1
    assert L.mgs_status_string(2) == b"MGS_ERANK"

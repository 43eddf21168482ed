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


def test_host_argument_checks_newton_and_batched(lib):
    """The Newton step and the batched solve reject bad arguments (including empty
    problems) on the host, before any CUDA call."""
    from paper_1210_0800_gb300 import _binding

    L = _binding.load()
    vp, c_double = ctypes.c_void_p, ctypes.c_double
    good = vp(4096)
    st = vp(8192)
    args = lambda J, ldj, x, m, n, tol: (J, ldj, good, x, m, n, c_double(tol), good, good, 1 << 20, st, None)
    assert L.newton_step_dd(*args(None, 4, good, 4, 4, 0.0)) == 1      # null J
    assert L.newton_step_dd(*args(good, 4, good, 3, 4, 0.0)) == 1      # m < n
    assert L.newton_step_qd(*args(good, 4, good, 4, 0, 0.0)) == 1      # n = 0 (empty)
    assert L.newton_step_d(*args(good, 2, good, 4, 4, 0.0)) == 1       # ldj < m
    assert L.newton_step_dd(*args(good, 4, good, 4, 4, -1.0)) == 1     # negative tolerance
    assert L.newton_step_dd(*args(good, 4, vp(4104), 4, 4, 0.0)) == 1  # misaligned x
    i64 = vp(4096)
    bargs = lambda batch, max_m, max_n, A: (A, good, good, None, i64, i64, i64, None, good, good, None, batch,
                                            max_m, max_n, good, 1 << 20, st, None, None)
    assert L.ls_solve_dd_batched(*bargs(0, 4, 4, good)) == 1           # empty batch
    assert L.ls_solve_qd_batched(*bargs(8, 3, 4, good)) == 1           # max_m < max_n
    assert L.ls_solve_d_batched(*bargs(8, 4, 4, vp(4104))) == 1        # misaligned pool


def test_host_argument_checks_wait_probe(lib):
    """The wait probe rejects bad arguments on the host, before any CUDA call."""
    from paper_1210_0800_gb300 import _binding

    L = _binding.load()
    vp = ctypes.c_void_p
    good, st = vp(4096), vp(8192)
    assert L.mgs_wait_probe(None, 0, 1000, st) == 1          # null words
    assert L.mgs_wait_probe(vp(4098), 0, 1000, st) == 1      # misaligned words
    assert L.mgs_wait_probe(good, 2, 1000, st) == 1          # unknown kind
    assert L.mgs_wait_probe(good, 1, 0, st) == 1             # no time limit
    assert L.mgs_wait_probe(good, 0, 20 * 10 ** 9, st) == 1  # above 10 s


def test_version_and_tune_struct(lib):
    """The version announces the mgs_tune layout the binding marshals (four ints)."""
    from paper_1210_0800_gb300 import _binding

    lib.mgs_version.restype = ctypes.c_int
    assert lib.mgs_version() == 200
    assert ctypes.sizeof(_binding.MgsTune) == 4 * ctypes.sizeof(ctypes.c_int)
    assert [f[0] for f in _binding.MgsTune._fields_] == ["threads", "ctas_per_sm", "split", "chunks"]

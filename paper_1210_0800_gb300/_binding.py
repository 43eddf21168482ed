"""ctypes binding of the C ABI (include/mgs_ddqd.h): argument marshalling only.

Every step of the solve runs in the CUDA library; there is no CPU path.  Tensors are
PyTorch float64 CUDA tensors in the layout of ``paper_1210_0800_gb300.inputs``:
a matrix (n, m, 2, L) column-major by element, a vector (m, 2, L).
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

MGS_OK, MGS_EINVAL, MGS_ERANK, MGS_ENONFINITE, MGS_ETIMEOUT, MGS_ECUDA, MGS_ENOSPACE = range(7)
STATUS_NAMES = {0: "MGS_OK", 1: "MGS_EINVAL", 2: "MGS_ERANK", 3: "MGS_ENONFINITE", 4: "MGS_ETIMEOUT",
                5: "MGS_ECUDA", 6: "MGS_ENOSPACE"}

EXPORTS = ["mgs_version", "mgs_status_string", "mgs_last_cuda_error", "mgs_workspace_bytes",
           "mgs_qr_dd", "mgs_qr_qd", "ls_solve_dd", "ls_solve_qd", "ls_solve_dd_noalloc"]

_lib = None


class MGSError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s: %s" % (what, STATUS_NAMES.get(code, code)))


def library_path() -> str:
    return _build.LIBRARY


def load(path: str | None = None):
    """Load the CUDA library; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIBRARY
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run paper_1210_0800_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i, sz, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
    lib.mgs_version.restype = i
    lib.mgs_status_string.restype = ctypes.c_char_p
    lib.mgs_status_string.argtypes = [i]
    lib.mgs_last_cuda_error.restype = i
    lib.mgs_workspace_bytes.restype = sz
    lib.mgs_workspace_bytes.argtypes = [i, i, i, i]
    qr_args = [dp, i, dp, i, i, i, vp, sz, vp, vp]
    ls_args = [dp, i, dp, dp, dp, i, dp, i, i, vp, sz, vp, vp]
    for name in ("mgs_qr_dd", "mgs_qr_qd"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = qr_args
    for name in ("ls_solve_dd", "ls_solve_qd"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = ls_args
    lib.ls_solve_dd_noalloc.restype = i
    lib.ls_solve_dd_noalloc.argtypes = [dp, i, dp, dp, dp, i, dp, i, i, vp, vp]
    if path == _build.LIBRARY:
        _lib = lib
    return lib


def _check_tensor(t, L, ndim_shape, name):
    import torch

    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if t.shape[-2:] != (2, L) or t.dim() != ndim_shape:
        raise ValueError("%s has shape %s; expected (..., 2, %d)" % (name, tuple(t.shape), L))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_bytes(limbs: int, m: int, n: int, with_rhs: bool) -> int:
    return int(load().mgs_workspace_bytes(limbs, m, n, 1 if with_rhs else 0))


def _workspace(limbs, m, n, with_rhs, device, workspace):
    import torch

    need = workspace_bytes(limbs, m, n, with_rhs)
    if need == 0:
        raise MGSError(MGS_ENOSPACE, "unsupported problem size m=%d n=%d" % (m, n))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    return workspace, need


def _ls_solve(limbs, A, b, x=None, R=None, z=None, workspace=None, status=None, stream=None):
    import torch

    n, m = A.shape[0], A.shape[1]
    _check_tensor(A, limbs, 4, "A")
    _check_tensor(b, limbs, 3, "b")
    if b.shape[0] != m:
        raise ValueError("b has %d rows, A has %d" % (b.shape[0], m))
    if x is None:
        x = torch.empty((n, 2, limbs), dtype=torch.float64, device=A.device)
    _check_tensor(x, limbs, 3, "x")
    if R is not None:
        _check_tensor(R, limbs, 4, "R")
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=A.device)
    ws, need = _workspace(limbs, m, n, True, A.device, workspace)
    fn = load().ls_solve_dd if limbs == 2 else load().ls_solve_qd
    rc = fn(_ptr(A), m, _ptr(b), _ptr(x), _ptr(R), n, _ptr(z), m, n, _ptr(ws), ctypes.c_size_t(ws.numel()),
            _ptr(status), _stream(stream))
    if rc != MGS_OK:
        extra = " (cudaError %d)" % load().mgs_last_cuda_error() if rc == MGS_ECUDA else ""
        raise MGSError(rc, "ls_solve%s" % extra)
    return x, status


def _mgs_qr(limbs, A, R=None, workspace=None, status=None, stream=None):
    import torch

    n, m = A.shape[0], A.shape[1]
    _check_tensor(A, limbs, 4, "A")
    if R is None:
        R = torch.zeros((n, n, 2, limbs), dtype=torch.float64, device=A.device)
    _check_tensor(R, limbs, 4, "R")
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=A.device)
    ws, need = _workspace(limbs, m, n, False, A.device, workspace)
    fn = load().mgs_qr_dd if limbs == 2 else load().mgs_qr_qd
    rc = fn(_ptr(A), m, _ptr(R), n, m, n, _ptr(ws), ctypes.c_size_t(ws.numel()), _ptr(status), _stream(stream))
    if rc != MGS_OK:
        extra = " (cudaError %d)" % load().mgs_last_cuda_error() if rc == MGS_ECUDA else ""
        raise MGSError(rc, "mgs_qr%s" % extra)
    return R, status


def ls_solve_dd(A, b, x=None, R=None, z=None, workspace=None, status=None, stream=None):
    """Complex DD least squares (MGS on [A b], back substitution); A -> Q, b -> residual."""
    return _ls_solve(2, A, b, x, R, z, workspace, status, stream)


def ls_solve_qd(A, b, x=None, R=None, z=None, workspace=None, status=None, stream=None):
    """Complex QD least squares (MGS on [A b], back substitution); A -> Q, b -> residual."""
    return _ls_solve(4, A, b, x, R, z, workspace, status, stream)


def ls_solve_dd_noalloc(A, b, x=None, R=None, z=None, status=None, stream=None):
    """ls_solve_dd with the library's built-in scratch array instead of a workspace, for
    callers that cannot allocate device memory (the outputs x and status must still be
    given, or are created here for convenience).  Calls that may overlap on the GPU race."""
    import torch

    n, m = A.shape[0], A.shape[1]
    _check_tensor(A, 2, 4, "A")
    _check_tensor(b, 2, 3, "b")
    if x is None:
        x = torch.empty((n, 2, 2), dtype=torch.float64, device=A.device)
    _check_tensor(x, 2, 3, "x")
    if R is not None:
        _check_tensor(R, 2, 4, "R")
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=A.device)
    rc = load().ls_solve_dd_noalloc(_ptr(A), m, _ptr(b), _ptr(x), _ptr(R), n, _ptr(z), m, n, _ptr(status),
                                    _stream(stream))
    if rc != MGS_OK:
        extra = " (cudaError %d)" % load().mgs_last_cuda_error() if rc == MGS_ECUDA else ""
        raise MGSError(rc, "ls_solve_dd_noalloc%s" % extra)
    return x, status


def mgs_qr_dd(A, R=None, workspace=None, status=None, stream=None):
    """Complex DD modified Gram-Schmidt QR; A -> Q in place, returns (R, status)."""
    return _mgs_qr(2, A, R, workspace, status, stream)


def mgs_qr_qd(A, R=None, workspace=None, status=None, stream=None):
    """Complex QD modified Gram-Schmidt QR; A -> Q in place, returns (R, status)."""
    return _mgs_qr(4, A, R, workspace, status, stream)


def mgs_workspace_bytes(limbs: int, m: int, n: int, with_rhs: bool = True) -> int:
    return workspace_bytes(limbs, m, n, with_rhs)

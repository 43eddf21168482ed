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
           "mgs_qr_dd", "mgs_qr_qd", "ls_solve_dd", "ls_solve_qd", "ls_solve_dd_noalloc",
           "mgs_batched_workspace_bytes", "ls_solve_dd_batched", "ls_solve_qd_batched",
           "ls_adjoint_dd_batched", "ls_adjoint_qd_batched", "mgs_qr_d", "ls_solve_d", "ls_solve_d_batched", "mgs_plan_query",
           "newton_workspace_bytes", "newton_step_d", "newton_step_dd", "newton_step_qd", "mgs_fp64_probe",
           "mgs_wait_probe"]


class MgsTune(ctypes.Structure):
    """Launch shape of the batched solve (mgs_tune in the C header)."""
    _fields_ = [("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("split", ctypes.c_int),
                ("chunks", ctypes.c_int)]

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
    lib.newton_workspace_bytes.restype = sz
    lib.newton_workspace_bytes.argtypes = [i, i, i]
    for name in ("newton_step_d", "newton_step_dd", "newton_step_qd"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = [dp, i, dp, dp, i, i, ctypes.c_double, vp, vp, sz, vp, vp]
    lib.mgs_fp64_probe.restype = i
    lib.mgs_fp64_probe.argtypes = [dp, i, i, i, vp]
    lib.mgs_wait_probe.restype = i
    lib.mgs_wait_probe.argtypes = [vp, i, ctypes.c_longlong, vp]
    lib.mgs_plan_query.restype = i
    lib.mgs_plan_query.argtypes = [i, i, i, i, ctypes.POINTER(ctypes.c_int)]
    qr_args = [dp, i, dp, i, i, i, vp, sz, vp, vp]
    ls_args = [dp, i, dp, dp, dp, i, dp, i, i, vp, sz, vp, vp]
    for name in ("mgs_qr_d", "mgs_qr_dd", "mgs_qr_qd"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = qr_args
    for name in ("ls_solve_d", "ls_solve_dd", "ls_solve_qd"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = ls_args
    lib.ls_solve_dd_noalloc.restype = i
    lib.ls_solve_dd_noalloc.argtypes = [dp, i, dp, dp, dp, i, dp, i, i, vp, vp]
    tp = ctypes.POINTER(MgsTune)
    lib.mgs_batched_workspace_bytes.restype = sz
    lib.mgs_batched_workspace_bytes.argtypes = [i, i, i, i, tp]
    for name in ("ls_solve_d_batched", "ls_solve_dd_batched", "ls_solve_qd_batched"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = [dp, dp, dp, dp, vp, vp, vp, vp, vp, vp, vp, i, i, i, vp, sz, vp, tp, vp]
    for name in ("ls_adjoint_dd_batched", "ls_adjoint_qd_batched"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = [dp, dp, dp, dp, dp, dp, dp, vp, vp, vp, vp, vp, vp, vp, i, i, i, vp, sz, vp,
                                       tp, vp]
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
    fn = {1: load().ls_solve_d, 2: load().ls_solve_dd, 4: load().ls_solve_qd}[limbs]
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
    fn = {1: load().mgs_qr_d, 2: load().mgs_qr_dd, 4: load().mgs_qr_qd}[limbs]
    rc = fn(_ptr(A), m, _ptr(R), n, m, n, _ptr(ws), ctypes.c_size_t(ws.numel()), _ptr(status), _stream(stream))
    if rc != MGS_OK:
        extra = " (cudaError %d)" % load().mgs_last_cuda_error() if rc == MGS_ECUDA else ""
        raise MGSError(rc, "mgs_qr%s" % extra)
    return R, status


def ls_solve_d(A, b, x=None, R=None, z=None, workspace=None, status=None, stream=None):
    """Complex double least squares (the paper's plain complex double runs)."""
    return _ls_solve(1, A, b, x, R, z, workspace, status, stream)


def mgs_qr_d(A, R=None, workspace=None, status=None, stream=None):
    """Complex double modified Gram-Schmidt QR; A -> Q in place, returns (R, status)."""
    return _mgs_qr(1, A, R, workspace, status, stream)


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


def fp64_probe(blocks: int, threads: int = 256, iters: int = 4096, reps: int = 5) -> float:
    """Measured FP64 fused multiply-add lane-operations per second of this GPU (the best of
    `reps` timed launches of mgs_fp64_probe)."""
    import torch

    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    best = 0.0
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = load().mgs_fp64_probe(_ptr(out), blocks, threads, iters, _stream(st))
        e1.record(st)
        if rc != MGS_OK:
            raise MGSError(rc, "mgs_fp64_probe")
        torch.cuda.synchronize()
        if r:  # the first launch warms up
            best = max(best, blocks * threads * iters * 8 / (e0.elapsed_time(e1) / 1000.0))
    return best


def mgs_wait_probe(words, kind: int, timeout_s: float) -> float:
    """Run one of the solver's bounded waits until it runs out (kind 0: the pivot-flag wait,
    kind 1: the grid barrier; `words`: 4 int32 device words, see the C header); returns the
    kernel's duration in seconds (CUDA events).  The status is left in words[2]."""
    import torch

    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    rc = load().mgs_wait_probe(_ptr(words), int(kind), int(timeout_s * 1e9), _stream(st))
    e1.record(st)
    if rc != MGS_OK:
        raise MGSError(rc, "mgs_wait_probe")
    e1.synchronize()
    return e0.elapsed_time(e1) / 1000.0


def mgs_plan_query(limbs: int, m: int, n: int, with_rhs: bool = True) -> dict:
    """Layout of a single-system call on the current device: row blocks Br, column groups
    Bc, rows per block h, the kernel ("grid", "cluster" or "group") and threads per CTA."""
    out = (ctypes.c_int * 5)()
    rc = load().mgs_plan_query(limbs, m, n, 1 if with_rhs else 0, out)
    if rc != 0:
        raise MGSError(rc, "mgs_plan_query")
    return dict(Br=out[0], Bc=out[1], h=out[2], kernel=("grid", "cluster", "group")[out[3]], threads=out[4])


# ----------------------------------------------------------------------------- batched


class Batch:
    """Device pools and index arrays of a ragged batch of least-squares systems.

    A_pool (sum m_i n_i, 2, L), b_pool (sum m_i, 2, L), x_pool (sum n_i, 2, L), element
    offsets a_off/b_off/x_off (int64), sizes m/n (int32), all on one CUDA device."""

    def __init__(self, A_pool, b_pool, x_pool, a_off, b_off, x_off, m, n, max_m, max_n, order=None, R_pool=None,
                 r_off=None):
        self.A_pool, self.b_pool, self.x_pool = A_pool, b_pool, x_pool
        self.a_off, self.b_off, self.x_off, self.m, self.n = a_off, b_off, x_off, m, n
        self.max_m, self.max_n, self.order = max_m, max_n, order
        self.R_pool, self.r_off = R_pool, r_off  # optional packed-R output
        self.batch = int(m.numel())
        self.limbs = int(A_pool.shape[-1])

    def set_order(self, kind):
        """Set the hand-out order of the work queue (see batch_order); returns self."""
        import torch

        ords = batch_order(self.m.cpu().numpy(), self.n.cpu().numpy(), kind)
        self.order = None if ords is None else torch.from_numpy(ords).to(self.A_pool.device)
        return self

    def with_R(self):
        """Allocate the packed-R output pool (n(n+1)/2 elements per system)."""
        import torch

        ns = self.n.to(torch.int64)
        sizes = ns * (ns + 1) // 2
        self.r_off = torch.cumsum(sizes, 0) - sizes
        self.R_pool = torch.zeros((int(sizes.sum().item()), 2, self.limbs), dtype=torch.float64,
                                  device=self.A_pool.device)
        return self


def batch_order(ms, ns, kind):
    """The order in which the work queue hands the systems out (an int32 permutation, or
    None for 0, 1, 2, ...).  "largest": decreasing m n^2, which balances the end of the
    launch; "interleave": the largest and the smallest alternately (largest, smallest,
    second largest, ...), so the first wave holds about half the bytes of the largest-first
    one and fits L2 better, and the queue still ends on middle-sized systems."""
    import numpy as np

    if kind is None or kind == "natural":
        return None
    work = np.asarray(ms, dtype=np.float64) * np.asarray(ns, dtype=np.float64) ** 2
    desc = np.argsort(-work, kind="stable").astype(np.int32)
    if kind == "largest":
        return desc
    if kind == "interleave":
        out = np.empty_like(desc)
        out[0::2] = desc[:(len(desc) + 1) // 2]
        out[1::2] = desc[::-1][:len(desc) // 2]
        return out
    raise ValueError("unknown order %r" % (kind,))


def make_batch(systems, device, largest_first=True, order=None):
    """Pack a list of (A (n, m, 2, L), b (m, 2, L)) numpy systems into a Batch (copies to
    the device).  order: "largest", "interleave" or "natural" (see batch_order); without
    it, largest_first=True means "largest" and False "natural"."""
    import numpy as np
    import torch

    L = systems[0][0].shape[-1]
    ms = np.array([A.shape[1] for A, _ in systems], dtype=np.int32)
    ns = np.array([A.shape[0] for A, _ in systems], dtype=np.int32)
    a_off = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(ms.astype(np.int64))[:-1]]).astype(np.int64)
    x_off = np.concatenate([[0], np.cumsum(ns.astype(np.int64))[:-1]]).astype(np.int64)
    A_pool = np.concatenate([A.reshape(-1, 2, L) for A, _ in systems])
    b_pool = np.concatenate([b.reshape(-1, 2, L) for _, b in systems])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    kind = order if order is not None else ("largest" if largest_first else "natural")
    ords = batch_order(ms, ns, kind)
    x_pool = torch.zeros((int(ns.sum()), 2, L), dtype=torch.float64, device=device)
    return Batch(t(A_pool), t(b_pool), x_pool, t(a_off), t(b_off), t(x_off), t(ms), t(ns),
                 int(ms.max()), int(ns.max()), None if ords is None else t(ords))


def batched_workspace_bytes(limbs, batch, max_m, max_n, tune=None):
    tp = ctypes.byref(MgsTune(*tune)) if tune else None
    return int(load().mgs_batched_workspace_bytes(limbs, batch, max_m, max_n, tp))


def ls_solve_batched(bt, workspace=None, status=None, tune=None, stream=None):
    """Solve every system of Batch `bt` in one launch (A -> Q, b -> residual, x filled).
    tune = (threads, ctas_per_sm[, split[, chunks]]) or None.  Returns the per-system
    status tensor."""
    import torch

    L = bt.limbs
    dev = bt.A_pool.device
    need = batched_workspace_bytes(L, bt.batch, bt.max_m, bt.max_n, tune)
    if need == 0:
        raise MGSError(MGS_ENOSPACE, "unsupported batch shape")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    if status is None:
        status = torch.empty(bt.batch, dtype=torch.int32, device=dev)
    fn = {1: load().ls_solve_d_batched, 2: load().ls_solve_dd_batched, 4: load().ls_solve_qd_batched}[L]
    tp = ctypes.byref(MgsTune(*tune)) if tune else None
    rc = fn(_ptr(bt.A_pool), _ptr(bt.b_pool), _ptr(bt.x_pool), _ptr(bt.R_pool), _ptr(bt.a_off), _ptr(bt.b_off),
            _ptr(bt.x_off), _ptr(bt.r_off), _ptr(bt.m), _ptr(bt.n), _ptr(bt.order), bt.batch, bt.max_m, bt.max_n,
            _ptr(workspace), ctypes.c_size_t(workspace.numel()), _ptr(status), tp, _stream(stream))
    if rc != MGS_OK:
        extra = " (cudaError %d)" % load().mgs_last_cuda_error() if rc == MGS_ECUDA else ""
        raise MGSError(rc, "ls_solve_batched%s" % extra)
    return status


def ls_solve_dd_batched(bt, workspace=None, status=None, tune=None, stream=None):
    assert bt.limbs == 2
    return ls_solve_batched(bt, workspace, status, tune, stream)


def ls_solve_qd_batched(bt, workspace=None, status=None, tune=None, stream=None):
    assert bt.limbs == 4
    return ls_solve_batched(bt, workspace, status, tune, stream)


def ls_adjoint_batched(bt, G_pool, gA_pool=None, gb_pool=None, workspace=None, status=None, tune=None, stream=None):
    """Gradients of a real loss through the batched solve already run on `bt` (which must
    hold Q in A_pool, the residual in b_pool, x in x_pool and the packed R).  G_pool is
    dL/dx laid out like x_pool.  Returns (gA_pool, gb_pool, status)."""
    import torch

    if bt.R_pool is None:
        raise ValueError("the forward solve must have produced R (Batch.with_R())")
    dev = bt.A_pool.device
    if gA_pool is None:
        gA_pool = torch.empty_like(bt.A_pool)
    if gb_pool is None:
        gb_pool = torch.empty_like(bt.b_pool)
    if workspace is None:
        workspace = torch.empty(256, dtype=torch.uint8, device=dev)
    if status is None:
        status = torch.empty(bt.batch, dtype=torch.int32, device=dev)
    if bt.limbs not in (2, 4):
        raise ValueError("the adjoint is built for complex double-double and quad-double (limbs 2 or 4)")
    fn = load().ls_adjoint_dd_batched if bt.limbs == 2 else load().ls_adjoint_qd_batched
    tp = ctypes.byref(MgsTune(*tune)) if tune else None
    rc = fn(_ptr(bt.A_pool), _ptr(bt.R_pool), _ptr(bt.x_pool), _ptr(bt.b_pool), _ptr(G_pool), _ptr(gA_pool),
            _ptr(gb_pool), _ptr(bt.a_off), _ptr(bt.r_off), _ptr(bt.b_off), _ptr(bt.x_off), _ptr(bt.m), _ptr(bt.n),
            _ptr(bt.order), bt.batch, bt.max_m, bt.max_n, _ptr(workspace), ctypes.c_size_t(workspace.numel()),
            _ptr(status), tp, _stream(stream))
    if rc != MGS_OK:
        extra = " (cudaError %d)" % load().mgs_last_cuda_error() if rc == MGS_ECUDA else ""
        raise MGSError(rc, "ls_adjoint_batched%s" % extra)
    return gA_pool, gb_pool, status

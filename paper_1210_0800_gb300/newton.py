"""Newton corrector on the device (Section 7): repeated least-squares solves of the
linearised system J(x) dx = -F(x) and updates x <- x + dx, with the stopping test and the
history kept in device memory so that a run needs one host read at its end.

The caller evaluates F and J = F' on the device (``evaluate(x, J, F)`` writes them into
the given tensors on the current stream); this package does not evaluate functions."""

from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as _b

HISTORY = 64
STATE_BYTES = 16 + 4 * 8 * HISTORY


class NewtonState:
    """Device copy of mgs_newton_state (include/mgs_ddqd.h)."""

    def __init__(self, device):
        import torch

        self.buf = torch.zeros(STATE_BYTES, dtype=torch.uint8, device=device)

    def reset(self):
        self.buf.zero_()

    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())

    def read(self) -> dict:
        raw = self.buf.cpu().numpy()
        head = raw[:16].view(np.int32)
        hist = raw[16:].view(np.float64).reshape(4, HISTORY)
        it = int(head[1])
        k = min(it, HISTORY)
        return dict(done=int(head[0]), iterations=it, status=int(head[2]), f_norm=hist[0, :k].copy(),
                    dx_norm=hist[1, :k].copy(), x_norm=hist[2, :k].copy(), z=hist[3, :k].copy())


def workspace_bytes(limbs: int, m: int, n: int) -> int:
    return int(_b.load().newton_workspace_bytes(limbs, m, n))


def newton_step(J, F, x, tol: float, state: NewtonState, workspace=None, status=None, stream=None):
    """One gated step (newton_step_d/dd/qd): J (n, m, 2, L) and F (m, 2, L) are consumed,
    x (n, 2, L) is updated in place unless the state says the run is over."""
    import torch

    L = x.shape[-1]
    n, m = J.shape[0], J.shape[1]
    _b._check_tensor(J, L, 4, "J")
    _b._check_tensor(F, L, 3, "F")
    _b._check_tensor(x, L, 3, "x")
    if F.shape[0] != m or x.shape[0] != n:
        raise ValueError("F must have m=%d rows and x n=%d entries" % (m, n))
    need = workspace_bytes(L, m, n)
    if need == 0:
        raise _b.MGSError(_b.MGS_ENOSPACE, "unsupported problem size m=%d n=%d" % (m, n))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=J.device)
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=J.device)
    fn = {1: _b.load().newton_step_d, 2: _b.load().newton_step_dd, 4: _b.load().newton_step_qd}[L]
    rc = fn(_b._ptr(J), m, _b._ptr(F), _b._ptr(x), m, n, ctypes.c_double(tol), state.ptr(), _b._ptr(workspace),
            ctypes.c_size_t(workspace.numel()), _b._ptr(status), _b._stream(stream))
    if rc != _b.MGS_OK:
        raise _b.MGSError(rc, "newton_step")
    return workspace, status


def newton_corrector(evaluate, x, m: int, tol: float = 1e-24, max_iter: int = 8, stream=None):
    """Run up to max_iter gated Newton steps from x (updated in place); returns the state
    read once at the end.  evaluate(x, J, F) is called before every step (also after the
    run has stopped: the gate skips only this package's kernels)."""
    import torch

    L = x.shape[-1]
    n = x.shape[0]
    J = torch.empty((n, m, 2, L), dtype=torch.float64, device=x.device)
    F = torch.empty((m, 2, L), dtype=torch.float64, device=x.device)
    state = NewtonState(x.device)
    ws, st = None, None
    for _ in range(max_iter):
        evaluate(x, J, F)
        ws, st = newton_step(J, F, x, tol, state, workspace=ws, status=st, stream=stream)
    return state.read()

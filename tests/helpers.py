"""Shared helpers of the GPU tests: run the CUDA path on numpy inputs, compare with the
oracle through its exact comparison routine."""

from __future__ import annotations

import math

import numpy as np

from paper_1210_0800_gb300 import inputs

TOL = {1: 1e-10, 2: 1e-26, 4: 1e-56}  # relative agreement with the oracle on well-conditioned inputs


def gpu_ls_solve(A: np.ndarray, b: np.ndarray, with_R: bool = True):
    import torch

    import paper_1210_0800_gb300 as mg

    n, m, _, L = A.shape
    dev = torch.device("cuda:0")
    At = torch.from_numpy(A).to(dev)
    bt = torch.from_numpy(b).to(dev)
    Rt = torch.zeros((n, n, 2, L), dtype=torch.float64, device=dev) if with_R else None
    zt = torch.zeros(L, dtype=torch.float64, device=dev)
    fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
    x, st = fn(At, bt, R=Rt, z=zt)
    torch.cuda.synchronize()
    out = dict(Q=At.cpu().numpy(), resid=bt.cpu().numpy(), x=x.cpu().numpy(), z=zt.cpu().numpy(),
               status=int(st.item()))
    if with_R:
        out["R"] = Rt.cpu().numpy()
    return out


def gpu_qr(A: np.ndarray):
    import torch

    import paper_1210_0800_gb300 as mg

    n, m, _, L = A.shape
    At = torch.from_numpy(A).to("cuda:0")
    fn = {1: mg.mgs_qr_d, 2: mg.mgs_qr_dd, 4: mg.mgs_qr_qd}[L]
    R, st = fn(At)
    torch.cuda.synchronize()
    return At.cpu().numpy(), R.cpu().numpy(), int(st.item())


def upper(R: np.ndarray) -> np.ndarray:
    """Copy of R (n, n, 2, L) with the strictly lower triangle zeroed (R[j, i] is (i, j))."""
    out = R.copy()
    n = R.shape[0]
    for j in range(n):
        out[j, j + 1:] = 0.0
    return out


def rel(orc, got, want) -> float:
    d, mx = orc.max_abs_diff(got, want)
    return d / mx if mx > 0 else d


def compare_ls(orc, A, b, tol=None):
    """GPU ls_solve vs oracle ls_solve on the same inputs: x, R, Q, z, residual."""
    L = A.shape[-1]
    tol = TOL[L] if tol is None else tol
    g = gpu_ls_solve(A.copy(), b.copy())
    o = orc.ls_solve(A.copy(), b.copy())
    assert g["status"] == 0 and o["status"] == 0, (g["status"], o["status"])
    errs = dict(
        x=rel(orc, g["x"], o["x"]),
        R=rel(orc, upper(g["R"]), upper(o["R"])),
        Q=rel(orc, g["Q"], o["Q"]),
        resid=orc.max_abs_diff(g["resid"], o["resid"])[0] / max(orc.max_abs_diff(b, 0 * b)[0], 1e-300),
        z=abs(float(np.sum(g["z"])) - float(np.sum(o["z"]))) / max(orc.max_abs_diff(b, 0 * b)[0], 1e-300),
    )
    for k, v in errs.items():
        assert v <= tol, (k, v, tol, A.shape)
    return errs, g, o


def planted_system(m, n, L, seed, extreme=False, orc=None):
    """A, x_true and b = A x_true (b formed exactly by the oracle, rounded to L limbs)."""
    A, xt, _ = inputs.system(m, n, L, seed, extreme=extreme)
    b = orc.matvec(A, xt)
    return A, xt, b


def kappa_estimate(orc, A, R):
    afro = math.sqrt(float(np.sum(A[..., 0] ** 2)))
    return afro * orc.rinv_fro(R)

"""Differentiable complex DD/QD least squares for uniform batches, as a
torch.autograd.Function around the batched solve and its adjoint kernel.

Tensors use the limb layout of the rest of the package: A (B, n, m, 2, L) (column-major
by element per system), b (B, m, 2, L), x (B, n, 2, L).  Gradients follow PyTorch's
convention for complex parameters, grad = dL/dRe + i dL/dIm, stored in the same limb
layout (as DD/QD numbers).  The forward keeps Q, R, x and the residual for the backward
when they fit the memory budget; otherwise it keeps A and b and the backward solves again.
"""

from __future__ import annotations

import torch

from . import _binding

DEFAULT_SAVE_BUDGET = 1 << 30  # bytes of saved factors above which Q, R are recomputed


def _uniform_batch(A, b):
    """Batch view of uniform systems (copies into fresh pools: the solve overwrites them)."""
    B, n, m, _, L = A.shape
    dev = A.device
    ar = torch.arange(B, device=dev, dtype=torch.int64)
    bt = _binding.Batch(A.reshape(B * n * m, 2, L).clone(), b.reshape(B * m, 2, L).clone(),
                        torch.zeros((B * n, 2, L), dtype=torch.float64, device=dev),
                        ar * (m * n), ar * m, ar * n,
                        torch.full((B,), m, dtype=torch.int32, device=dev),
                        torch.full((B,), n, dtype=torch.int32, device=dev), m, n)
    return bt.with_R()


def saved_bytes(B, m, n, L):
    return B * (m * n + n * (n + 1) // 2 + n + m) * 2 * L * 8


class LeastSquares(torch.autograd.Function):
    """x = argmin ||b - A x|| for every system of a uniform batch."""

    @staticmethod
    def forward(ctx, A, b, save_budget=DEFAULT_SAVE_BUDGET, tune=None):
        B, n, m, _, L = A.shape
        bt = _uniform_batch(A.detach(), b.detach())
        st = _binding.ls_solve_batched(bt, tune=tune)
        ctx.shape = (B, n, m, L)
        ctx.tune = tune
        ctx.recompute = saved_bytes(B, m, n, L) > save_budget
        if ctx.recompute:
            ctx.save_for_backward(A.detach(), b.detach())
        else:
            ctx.bt = bt
        ctx.status = st
        return bt.x_pool.reshape(B, n, 2, L)

    @staticmethod
    def backward(ctx, grad_x):
        B, n, m, L = ctx.shape
        if ctx.recompute:
            A, b = ctx.saved_tensors
            bt = _uniform_batch(A, b)
            _binding.ls_solve_batched(bt, tune=ctx.tune)
        else:
            bt = ctx.bt
        G = grad_x.contiguous().reshape(B * n, 2, L)
        gA, gb, _ = _binding.ls_adjoint_batched(bt, G, tune=ctx.tune)
        return gA.reshape(B, n, m, 2, L), gb.reshape(B, m, 2, L), None, None


def lstsq(A, b, save_budget=DEFAULT_SAVE_BUDGET, tune=None):
    """Differentiable batched least squares (see LeastSquares); complex double-double or
    quad-double (the last dimension of A and b holds 2 or 4 limbs)."""
    if A.shape[-1] not in (2, 4):
        raise ValueError("lstsq differentiates double-double and quad-double solves (2 or 4 limbs)")
    return LeastSquares.apply(A, b, save_budget, tune)

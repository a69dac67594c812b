"""``torch.autograd.Function`` over the differentiable FD entry points.

``fd_equalize(H, y, rho_c, nu, C)`` returns ``z`` (``[n_sc][n_sym][U]`` complex64)
of the FD architecture with per-cluster regularizers ``rho_c`` (``[C]``) and
fusion weights ``nu`` (``[C][U]``); its backward calls the hand-written adjoint
kernels (``ffeq_fd_train_backward``), which recompute the factorizations.
Gradients of complex tensors follow PyTorch's convention (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from . import ffeq


class FDEqualize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, y, rho_c, nu, C: int, precision: int = ffeq.FP32):
        H, y = H.contiguous(), y.contiguous()
        rho_c, nu = rho_c.contiguous().float(), nu.contiguous().float()
        n_sc, U, B = H.shape
        n_sym = y.shape[1]
        plan = ffeq.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ffeq.FD, precision=precision)
        nb = ffeq.ffeq_fd_train_workspace_size(plan)
        ws = torch.empty(nb, dtype=torch.uint8, device=H.device)
        z = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=H.device)
        ffeq.ffeq_fd_train_forward(plan, H, y, rho_c, nu, z, ws, nb)
        ctx.plan, ctx.ws, ctx.nb = plan, ws, nb
        ctx.save_for_backward(H, y, rho_c, nu)
        return z

    @staticmethod
    def backward(ctx, gz):
        H, y, rho_c, nu = ctx.saved_tensors
        gz = gz.contiguous().to(torch.complex64)
        gH = torch.empty_like(H)
        gy = torch.empty_like(y)
        grho = torch.empty_like(rho_c)
        gnu = torch.empty_like(nu)
        ffeq.ffeq_fd_train_backward(ctx.plan, H, y, rho_c, nu, gz, gH, gy, grho, gnu, ctx.ws, ctx.nb)
        return gH, gy, grho, gnu, None, None


def fd_equalize(H, y, rho_c, nu, C: int, precision: int = ffeq.FP32):
    """Differentiable FD equalization (see ``FDEqualize``)."""
    return FDEqualize.apply(H, y, rho_c, nu, C, precision)

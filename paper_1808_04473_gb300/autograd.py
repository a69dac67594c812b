"""``torch.autograd.Function`` over the differentiable FD entry points.

``fd_equalize(H, y, rho_c, nu, C)`` returns ``z`` (``[n_sc][n_sym][U]`` complex64)
of the FD architecture with per-cluster regularizers ``rho_c`` (``[C]``) and
fusion weights ``nu`` (``[C][U]``); its backward calls the hand-written adjoint
kernels (``ffeq_fd_train_backward``), which recompute the factorizations.

``fd_equalize_optimal(H, y, N0, Es, C)`` returns ``z`` of the FD architecture as
the paper defines it (unbiased L-MMSE pairs fused with the optimal weights of
Lemma 1, computed by ``ffeq_equalize``); its backward (``ffeq_fd_optimal_backward``)
differentiates through the weights' dependence on the local error variances.

Gradients of complex tensors follow PyTorch's convention (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from . import ffeq


class FDEqualize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, y, rho_c, nu, C: int, precision: int = ffeq.FP32, cluster_sizes=None):
        H, y = H.contiguous(), y.contiguous()
        rho_c, nu = rho_c.contiguous().float(), nu.contiguous().float()
        n_sc, U, B = H.shape
        n_sym = y.shape[1]
        plan = ffeq.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ffeq.FD, precision=precision,
                                     cluster_sizes=cluster_sizes)
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
        return gH, gy, grho, gnu, None, None, None


def fd_equalize(H, y, rho_c, nu, C: int, precision: int = ffeq.FP32, cluster_sizes=None):
    """Differentiable FD equalization (see ``FDEqualize``); ``cluster_sizes``: antennas
    per cluster (Sec. II-B), ``None`` for B / C each."""
    return FDEqualize.apply(H, y, rho_c, nu, C, precision, cluster_sizes)


class FDEqualizeOptimal(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, y, N0: float, Es: float, C: int, precision: int = ffeq.FP32, cluster_sizes=None):
        H, y = H.contiguous(), y.contiguous()
        n_sc, U, B = H.shape
        n_sym = y.shape[1]
        plan = ffeq.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ffeq.FD, precision=precision,
                                     cluster_sizes=cluster_sizes)
        nb = ffeq.ffeq_workspace_size(plan)
        ws = torch.empty(max(nb, 16), dtype=torch.uint8, device=H.device)
        z = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=H.device)
        s2 = torch.empty((n_sc, U), dtype=torch.float32, device=H.device)
        ffeq.ffeq_equalize(plan, H, y, N0, Es, z, s2, None, None, ws, nb)
        ctx.plan, ctx.N0, ctx.Es = plan, float(N0), float(Es)
        ctx.save_for_backward(H, y)
        return z

    @staticmethod
    def backward(ctx, gz):
        H, y = ctx.saved_tensors
        gz = gz.contiguous().to(torch.complex64)
        gH = torch.empty_like(H)
        gy = torch.empty_like(y)
        nb = ffeq.ffeq_fd_optimal_workspace_size(ctx.plan)
        ws = torch.empty(nb, dtype=torch.uint8, device=H.device)
        ffeq.ffeq_fd_optimal_backward(ctx.plan, H, y, ctx.N0, ctx.Es, gz, gH, gy, ws, nb)
        return gH, gy, None, None, None, None, None


def fd_equalize_optimal(H, y, N0: float, Es: float, C: int, precision: int = ffeq.FP32, cluster_sizes=None):
    """FD equalization with the paper's optimal fusion weights, differentiable in H and y
    (see ``FDEqualizeOptimal``)."""
    return FDEqualizeOptimal.apply(H, y, N0, Es, C, precision, cluster_sizes)

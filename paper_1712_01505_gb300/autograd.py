"""Differentiable pseudofermion action S = phi^dag (M^dag M)^-1 phi for the Wilson matrix.

M = 1 - kappa H is the hopping-parameter form of Eq. (1).  The forward pass solves
M^dag eta = phi and returns S = |eta|^2; the backward pass solves M X = eta afresh (the
Krylov history of the forward solve is not kept) and calls the outer-product link kernel:
dS = 2 kappa Re(eta^dag dH X), with the 18 reals of every link independent.  PyTorch's
complex gradient convention (dS/dRe + i dS/dIm) is what the kernel produces, and
dS/dphi = 2 (M^dag M)^-1 phi = 2 X.

All arithmetic runs in libqcd (qcd_solve, qcd_force); this module only moves tensors.
"""
from __future__ import annotations

import torch

from . import qcd


class WilsonPseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, kappa, L, bc=(1, 1, 1, -1), tol=1e-12, inner="f32"):
        if U.dtype != torch.complex128 or phi.dtype != torch.complex128:
            raise TypeError("U and phi must be complex128")
        if not (U.is_cuda and phi.is_cuda):
            raise ValueError("U and phi must be CUDA tensors")
        g = qcd.Gauge.load(U.detach().contiguous(), tuple(L), tuple(bc), recon=18)
        f = qcd.wilson(kappa)
        phi_c = phi.detach().contiguous()
        eta = torch.zeros_like(phi_c)
        qcd.solve(g, f, phi_c, eta, method=qcd.BICGSTAB, tol=tol, inner=inner, dagger=True)
        S = torch.tensor(qcd.norm2(g, f, eta)[0], dtype=torch.float64, device=phi.device)
        ctx.save_for_backward(eta)
        ctx.gauge, ctx.fermion, ctx.tol, ctx.inner = g, f, tol, inner
        ctx.shape_U = U.shape
        return S

    @staticmethod
    def backward(ctx, gS):
        (eta,) = ctx.saved_tensors
        g, f = ctx.gauge, ctx.fermion
        X = torch.zeros_like(eta)
        qcd.solve(g, f, eta, X, method=qcd.BICGSTAB, tol=ctx.tol, inner=ctx.inner)
        V = eta.shape[0]
        dS = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=eta.device)
        qcd.force(g, f, X, eta, dS)
        torch.cuda.current_stream().synchronize()
        gU = torch.view_as_complex(dS) * gS
        gphi = 2.0 * X * gS
        return gU.reshape(ctx.shape_U), gphi, None, None, None, None, None


def wilson_action(U, phi, kappa, L, bc=(1, 1, 1, -1), tol=1e-12, inner="f32"):
    """S = phi^dag (M^dag M)^-1 phi, differentiable in U (4, V, 3, 3) and phi (V, 4, 3)."""
    return WilsonPseudofermionAction.apply(U, phi, kappa, L, bc, tol, inner)

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


class WilsonEOPseudofermionAction(torch.autograd.Function):
    """S_eo = phi_e^dag (Mhat^dag Mhat)^-1 phi_e, Mhat = 1 - kappa^2 H_eo H_oe on the even sites.

    Forward: z = the even part of M^-dag (phi_e, 0) = Mhat^-dag phi_e, S = |z|^2.  Backward: X =
    the even part of M^-1 (z, 0) = (Mhat^dag Mhat)^-1 phi_e, then qcd_force_eo with Y = z
    (dS = 2 kappa^2 Re(eta^dag dH xi)); dS/dphi = 2 X on the even sites, 0 on the odd ones.
    """

    @staticmethod
    def forward(ctx, U, phi, kappa, L, bc=(1, 1, 1, -1), tol=1e-12, inner="f32"):
        if U.dtype != torch.complex128 or phi.dtype != torch.complex128:
            raise TypeError("U and phi must be complex128")
        if not (U.is_cuda and phi.is_cuda):
            raise ValueError("U and phi must be CUDA tensors")
        g = qcd.Gauge.load(U.detach().contiguous(), tuple(L), tuple(bc), recon=18)
        f = qcd.wilson(kappa)
        buf = torch.empty(qcd.field_bytes(g, f, "f64"), dtype=torch.uint8, device=phi.device)

        def even(src):  # src with its odd sites zeroed
            out = torch.zeros_like(src)
            qcd.field_pack(g, f, "f64", 0, src, buf)
            qcd.field_unpack(g, f, "f64", 0, buf, out)
            return out

        b = even(phi.detach().contiguous())
        w = torch.zeros_like(b)
        qcd.solve(g, f, b, w, method=qcd.BICGSTAB, tol=tol, inner=inner, dagger=True)
        z = even(w)
        S = torch.tensor(qcd.norm2(g, f, z)[0], dtype=torch.float64, device=phi.device)
        ctx.save_for_backward(z)
        ctx.gauge, ctx.fermion, ctx.tol, ctx.inner, ctx.even = g, f, tol, inner, even
        ctx.shape_U = U.shape
        return S

    @staticmethod
    def backward(ctx, gS):
        (z,) = ctx.saved_tensors
        g, f = ctx.gauge, ctx.fermion
        v = torch.zeros_like(z)
        qcd.solve(g, f, z, v, method=qcd.BICGSTAB, tol=ctx.tol, inner=ctx.inner)
        X = ctx.even(v)
        V = z.shape[0]
        dS = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=z.device)
        qcd.force_eo(g, f, X, z, dS)
        torch.cuda.current_stream().synchronize()
        gU = torch.view_as_complex(dS) * gS
        gphi = 2.0 * X * gS
        return gU.reshape(ctx.shape_U), gphi, None, None, None, None, None


def wilson_eo_action(U, phi, kappa, L, bc=(1, 1, 1, -1), tol=1e-12, inner="f32"):
    """S_eo = phi_e^dag (Mhat^dag Mhat)^-1 phi_e, differentiable in U (4, V, 3, 3) and phi (V, 4, 3)."""
    return WilsonEOPseudofermionAction.apply(U, phi, kappa, L, bc, tol, inner)

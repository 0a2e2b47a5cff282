"""Molecular dynamics of the even-odd Wilson pseudofermion action on the GPU.

Ensemble generation solves the fermion system many times (Sec. II A).  This module
integrates Hamilton's equations for

    H(U, P) = 1/2 sum_{x,mu} tr(P_mu(x)^dag P_mu(x)) + S_eo(U),
    S_eo(U) = phi_e^dag (Mhat^dag Mhat)^-1 phi_e,   Mhat = 1 - kappa^2 H_eo H_oe,

with dU/dt = P U and dP/dt = F, F = P_TA(U G^dag) the su(3) projection of the link
derivative G = dS/dRe U + i dS/dIm U (dH/dt = 0 for this pair), by the leapfrog
scheme.  Every force evaluation is two mixed-precision solves (qcd_solve with the
adjoint and with the plain operator, sources restricted to the even sites) followed by
qcd_force_eo and qcd_force_project; the integration steps are qcd_link_update and
qcd_mom_update, the kinetic term qcd_mom_energy.  The gauge action is not part of the
method's hot path and is left out: these dynamics move the links under the fermion
force alone.

All arithmetic runs in libqcd; this module allocates tensors and sequences calls.
"""
from __future__ import annotations

import torch

from . import qcd


class EOPseudofermionMD:
    """Leapfrog molecular dynamics for S_eo on a fixed lattice and pseudofermion field.

    phi: canonical (V, 4, 3) complex128 CUDA tensor (its odd sites are ignored).
    Solver keywords (tol, inner, outer, ...) go to qcd_solve.
    """

    def __init__(self, L, kappa, phi, bc=(1, 1, 1, -1), tol=1e-12, inner="f32", outer="df64", **solver):
        self.L, self.bc, self.kappa = tuple(L), tuple(bc), float(kappa)
        self.fermion = qcd.wilson(kappa)
        self.solver = dict(method=qcd.BICGSTAB, tol=tol, inner=inner, outer=outer, use_graph=True, **solver)
        self.phi = phi.contiguous()
        self.device = phi.device

    def _even(self, g, src):
        """A copy of src with its odd sites zeroed (pack the even sites, unpack into zeros)."""
        buf = torch.empty(qcd.field_bytes(g, self.fermion, "f64"), dtype=torch.uint8, device=self.device)
        out = torch.zeros_like(src)
        qcd.field_pack(g, self.fermion, "f64", 0, src, buf)
        qcd.field_unpack(g, self.fermion, "f64", 0, buf, out)
        return out

    def _solves(self, g):
        """S, X = (Mhat^dag Mhat)^-1 phi_e, Y = Mhat X (X, Y as full fields; their odd sites are
        not used): Y is the even part of M^-dag (phi_e, 0), X that of M^-1 (Y, 0)."""
        b = self._even(g, self.phi)
        w = torch.zeros_like(b)
        qcd.solve(g, self.fermion, b, w, dagger=True, **self.solver)
        z = self._even(g, w)
        S = qcd.norm2(g, self.fermion, z)[0]
        v = torch.zeros_like(b)
        qcd.solve(g, self.fermion, z, v, **self.solver)
        return S, v, z

    def action(self, U) -> float:
        g = qcd.Gauge.load(U, self.L, self.bc)
        try:
            return self._solves(g)[0]
        finally:
            g.free()

    def force(self, U, F=None):
        """F = P_TA(U G^dag) as (4, V, 3, 3) complex128; also returns S at U."""
        g = qcd.Gauge.load(U, self.L, self.bc)
        try:
            S, X, Y = self._solves(g)
            V = U.shape[1]
            dS = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=self.device)
            qcd.force_eo(g, self.fermion, X, Y, dS)
            if F is None:
                F = torch.empty((4, V, 3, 3), dtype=torch.complex128, device=self.device)
            qcd.force_project(g, dS, F)
            torch.cuda.current_stream(self.device).synchronize()
            return F, S
        finally:
            g.free()

    def hamiltonian(self, U, P) -> float:
        return 0.5 * qcd.mom_energy(P) + self.action(U)

    def leapfrog(self, U, P, eps, nsteps):
        """Advance (U, P) in place by nsteps leapfrog steps of size eps; returns (H_start, H_end)."""
        h0 = self.hamiltonian(U, P)
        F, _ = self.force(U)
        qcd.mom_update(P, F, 0.5 * eps)
        for k in range(nsteps):
            qcd.link_update(U, P, eps)
            self.force(U, F)
            qcd.mom_update(P, F, eps if k < nsteps - 1 else 0.5 * eps)
        torch.cuda.current_stream(self.device).synchronize()
        return h0, self.hamiltonian(U, P)

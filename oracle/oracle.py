"""FP64 CPU oracle: Python wrapper around ``qcd_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with the
GPU library (it never imports ``paper_1712_01505_gb300``) and the library never
imports it.

Every function takes and returns numpy ``complex128`` arrays in the canonical
layouts (see the header of ``qcd_oracle.c``):

* gauge field ``U``: ``(4, V, 3, 3)``; site index ``x + Lx*(y + Ly*(z + Lz*t))``
* 4D spinor: ``(V, 4, 3)``; 5D spinor: ``(Ls, V, 4, 3)``

Operators follow Kanamori & Matsufuru (arXiv:1712.01505): the Wilson matrix of
Eq. (1) in hopping-parameter form ``M = 1 - kappa H`` (``kappa = 1/(2(m0+4))``),
the domain-wall matrix of Eq. (2), BiCGStab for Wilson and CG on the normal
equations for domain-wall (Sec. II C).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

c_int_p = ctypes.POINTER(ctypes.c_int)
c_dbl_p = ctypes.POINTER(ctypes.c_double)
c_long_p = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile ``qcd_oracle.c`` into ``liboracle.so`` with gcc (FP64, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.ora_wilson_solve.restype = ctypes.c_long
        _lib.ora_dw_solve.restype = ctypes.c_long
        _lib.ora_num_threads.restype = ctypes.c_int
    return _lib


def _iarr(v):
    a = (ctypes.c_int * 4)(*[int(t) for t in v])
    return a


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    return lib().ora_num_threads()


def set_num_threads(n: int) -> None:
    """Threads used by the following oracle calls (timing only; results do not depend on it)."""
    lib().ora_set_num_threads(int(n))


def gamma(k: int) -> np.ndarray:
    """Dirac matrix gamma_{k+1} for k = 0..3, gamma_5 for k = 4 (chiral basis)."""
    out = np.zeros((4, 4, 2), dtype=np.float64)
    lib().ora_gamma(int(k), out.ctypes.data_as(c_dbl_p))
    return out[..., 0] + 1j * out[..., 1]


def volume(L) -> int:
    return int(np.prod(L))


def parity(L) -> np.ndarray:
    """Parity (x+y+z+t) mod 2 of every canonical site."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    return ((x + y + z + t) & 1).reshape(-1)


def hop(L, bc, U, psi, dagger=False, out_parity=-1):
    """H psi (Eq. (1) hopping term), or H^dag psi; optionally only on one parity."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    lib().ora_hop(_iarr(L), _iarr(bc), _p(U), _p(psi), _p(out), int(dagger), int(out_parity))
    return out


def hop_sites(L, bc, U, psi, sites, dagger=False):
    """(H psi)(x) at the canonical sites listed; returns (n, 4, 3)."""
    U, psi = _c(U), _c(psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    lib().ora_hop_sites(_iarr(L), _iarr(bc), _p(U), _p(psi), _p(sites), ctypes.c_long(len(sites)),
                        _p(out), int(dagger))
    return out


def wilson(L, bc, kappa, U, psi, dagger=False):
    """M psi with M = 1 - kappa H, or M^dag psi."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    lib().ora_wilson(_iarr(L), _iarr(bc), ctypes.c_double(kappa), _p(U), _p(psi), _p(out),
                     int(dagger))
    return out


def wilson_mhat(L, bc, kappa, U, psi_even, dagger=False):
    """Schur operator Mhat = 1 - kappa^2 H_eo H_oe on a full-lattice vector living on even sites."""
    U, psi = _c(U), _c(psi_even)
    out = np.empty_like(psi)
    lib().ora_wilson_mhat(_iarr(L), _iarr(bc), ctypes.c_double(kappa), _p(U), _p(psi), _p(out),
                          int(dagger))
    return out


def wilson_solve(L, bc, kappa, U, b, tol=1e-10, maxiter=100000, dagger=False):
    """Solve M x = b (or M^dag x = b); returns (x, iterations, full relative residual)."""
    U, b = _c(U), _c(b)
    x = np.zeros_like(b)
    res = ctypes.c_double(0)
    it = lib().ora_wilson_solve(_iarr(L), _iarr(bc), ctypes.c_double(kappa), _p(U), _p(b), _p(x),
                                ctypes.c_double(tol), ctypes.c_long(maxiter), int(dagger),
                                ctypes.byref(res))
    return x, int(it), res.value


def dw(L, bc, Ls, M5, mf, U, psi, dagger=False):
    """D_DW psi of Eq. (2) (or its adjoint) on a (Ls, V, 4, 3) field."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    lib().ora_dw(_iarr(L), _iarr(bc), int(Ls), ctypes.c_double(M5), ctypes.c_double(mf), _p(U),
                 _p(psi), _p(out), int(dagger))
    return out


def dw_block(Ls, V, M5, mf, psi, dagger=False):
    """A psi: the site-local (s, spin) part of Eq. (2)."""
    psi = _c(psi)
    out = np.empty_like(psi)
    lib().ora_dw_block_apply(int(Ls), ctypes.c_long(V), ctypes.c_double(M5), ctypes.c_double(mf),
                             _p(psi), _p(out), int(dagger))
    return out


def dw_ainv(Ls, V, M5, mf, psi, dagger=False):
    """A^-1 psi (A^-dag psi) by Gauss-Jordan inversion of the site-local block."""
    psi = _c(psi)
    out = np.empty_like(psi)
    lib().ora_dw_ainv(int(Ls), ctypes.c_long(V), ctypes.c_double(M5), ctypes.c_double(mf),
                      _p(psi), _p(out), int(dagger))
    return out


def dw_mhat(L, bc, Ls, M5, mf, U, psi_even, dagger=False):
    """Domain-wall Schur operator Mhat = 1 - 1/4 A^-1 H_eo A^-1 H_oe (or its adjoint)."""
    U, psi = _c(U), _c(psi_even)
    out = np.empty_like(psi)
    lib().ora_dw_mhat(_iarr(L), _iarr(bc), int(Ls), ctypes.c_double(M5), ctypes.c_double(mf),
                      _p(U), _p(psi), _p(out), int(dagger))
    return out


def dw_solve(L, bc, Ls, M5, mf, U, b, tol=1e-10, maxiter=100000):
    """Solve D_DW x = b by even-odd CG on Mhat^dag Mhat; returns (x, iterations, residual)."""
    U, b = _c(U), _c(b)
    x = np.zeros_like(b)
    res = ctypes.c_double(0)
    it = lib().ora_dw_solve(_iarr(L), _iarr(bc), int(Ls), ctypes.c_double(M5),
                            ctypes.c_double(mf), _p(U), _p(b), _p(x), ctypes.c_double(tol),
                            ctypes.c_long(maxiter), ctypes.byref(res))
    return x, int(it), res.value


def wilson_force(L, bc, kappa, X, eta):
    """dS/dU for S = phi^dag (M^dag M)^-1 phi given X = M^-1 eta, eta = M^-dag phi.

    Returns a (4, V, 3, 3, 2) float64 array: d S / d Re U_ab and d S / d Im U_ab.
    """
    X, eta = _c(X), _c(eta)
    V = volume(L)
    out = np.empty((4, V, 3, 3, 2), dtype=np.float64)
    lib().ora_wilson_force(_iarr(L), _iarr(bc), ctypes.c_double(kappa), _p(X), _p(eta), _p(out))
    return out


def wilson_action(L, bc, kappa, U, phi, tol=1e-13):
    """S = phi^dag (M^dag M)^-1 phi = |M^-dag phi|^2 and the solves behind it.

    Returns (S, eta, X).
    """
    eta, _, _ = wilson_solve(L, bc, kappa, U, phi, tol=tol, dagger=True)
    X, _, _ = wilson_solve(L, bc, kappa, U, eta, tol=tol, dagger=False)
    return float(np.vdot(eta, eta).real), eta, X


# ----------------------------------------------------------------------------- molecular dynamics
# Ensemble generation needs the solver many times (Sec. II A).  The pieces below
# are the molecular-dynamics ingredients for the even-odd pseudofermion action,
# written from their definitions: S_eo = phi_e^dag (Mhat^dag Mhat)^-1 phi_e with
# Mhat = 1 - kappa^2 H_eo H_oe, momenta P in su(3), U(t) = exp(t P) U.

def wilson_eo_action(L, bc, kappa, U, phi_e, tol=1e-13):
    """S_eo = phi_e^dag (Mhat^dag Mhat)^-1 phi_e for the even sites of phi_e (odd sites ignored).

    Uses the Schur complement of M = 1 - kappa H on the even sites: for b = (b_e, 0), the even
    part of M^-1 b is Mhat^-1 b_e (and of M^-dag b, Mhat^-dag b_e).  Returns (S, X, Y) with
    z = Mhat^-dag phi_e, X = Mhat^-1 z = (Mhat^dag Mhat)^-1 phi_e, Y = Mhat X = z, as canonical
    fields that vanish on the odd sites.
    """
    par = parity(L)
    b = _c(phi_e).copy()
    b[par == 1] = 0
    w, _, _ = wilson_solve(L, bc, kappa, U, b, tol=tol, dagger=True)
    z = w.copy()
    z[par == 1] = 0
    v, _, _ = wilson_solve(L, bc, kappa, U, z, tol=tol, dagger=False)
    X = v.copy()
    X[par == 1] = 0
    return float(np.vdot(z, z).real), X, z


def wilson_eo_force(L, bc, kappa, U, X, Y):
    """dS_eo/dU (4, V, 3, 3, 2) for X = (Mhat^dag Mhat)^-1 phi_e, Y = Mhat X.

    dS_eo = -2 Re(Y^dag dMhat X) with dMhat = -kappa^2 (dH_eo H_oe + H_eo dH_oe), i.e.
    2 kappa^2 Re(eta^dag dH xi) with xi = (X_e, H_oe X_e) and eta = (Y_e, (H^dag)_oe Y_e);
    ``wilson_force`` gives 2 kappa Re(eta^dag dH xi).
    """
    par = parity(L)
    Xe, Ye = _c(X).copy(), _c(Y).copy()
    Xe[par == 1] = 0
    Ye[par == 1] = 0
    xi = Xe + hop(L, bc, U, Xe, out_parity=1)
    eta = Ye + hop(L, bc, U, Ye, dagger=True, out_parity=1)
    return kappa * wilson_force(L, bc, kappa, xi, eta)


def su3_project(U, dSdU):
    """F = P_TA(U G^dag), G = dS/dRe U + i dS/dIm U; P_TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6."""
    U = _c(U)
    G = dSdU[..., 0] + 1j * dSdU[..., 1]
    M = U @ np.conj(np.swapaxes(G, -1, -2))
    A = 0.5 * (M - np.conj(np.swapaxes(M, -1, -2)))
    tr = np.trace(A, axis1=-2, axis2=-1) / 3.0
    return A - tr[..., None, None] * np.eye(3)


def link_update(U, P, eps):
    """U <- exp(eps P) U for every link (matrix exponential by scipy)."""
    from scipy.linalg import expm

    return expm(eps * _c(P)) @ _c(U)


def kinetic(P):
    """sum over links of tr(P^dag P) = sum |P_ab|^2."""
    return float(np.sum(np.abs(P) ** 2))


def leapfrog(L, bc, kappa, U, P, phi_e, eps, nsteps, tol=1e-13):
    """Leapfrog for H = K/2 + S_eo with K = sum tr(P^dag P) and dU/dt = P U, so that dH/dt = 0
    needs dP/dt = F = P_TA(U G^dag) (the derivative of S along P U is Re tr(P F)).
    Returns (U, P, H_start, H_end)."""
    def force(U):
        _, X, Y = wilson_eo_action(L, bc, kappa, U, phi_e, tol=tol)
        return su3_project(U, wilson_eo_force(L, bc, kappa, U, X, Y))

    def ham(U, P):
        return 0.5 * kinetic(P) + wilson_eo_action(L, bc, kappa, U, phi_e, tol=tol)[0]

    U, P = _c(U).copy(), _c(P).copy()
    h0 = ham(U, P)
    P = P + 0.5 * eps * force(U)
    for k in range(nsteps):
        U = link_update(U, P, eps)
        P = P + (eps if k < nsteps - 1 else 0.5 * eps) * force(U)
    return U, P, h0, ham(U, P)


# ----------------------------------------------------------------------------- Mobius domain-wall
# The Mobius generalisation of Eq. (2) (Brower, Neff and Orginos): with the fifth-dimension
# shift (S psi)_s = P_- psi_{s+1} + P_+ psi_{s-1} (factor -mf across the wall) and
# D_W = (4 - M5) - H/2 the 4D Wilson matrix of mass -M5,
#   D_M psi_s = (b5 D_W + 1) psi_s - (1 - c5 D_W) (S psi)_s = A psi - 1/2 H (B psi),
#   B = b5 + c5 S,   A = (4 - M5) B + 1 - S.
# b5 = 1, c5 = 0 is Eq. (2).  A and B act on (s, spin) at every site and colour.

def mobius_blocks(Ls, M5, mf, b5, c5):
    """A and B as (Ls, 4, Ls, 4) real arrays [s, spin, s', spin']."""
    Pp = np.diag([1.0, 1.0, 0.0, 0.0])  # (1 + gamma5)/2, gamma5 = diag(1, 1, -1, -1)
    Pm = np.diag([0.0, 0.0, 1.0, 1.0])
    S = np.zeros((Ls, 4, Ls, 4))
    for s in range(Ls):
        S[s, :, (s + 1) % Ls, :] += Pm * (-mf if s == Ls - 1 else 1.0)
        S[s, :, (s - 1) % Ls, :] += Pp * (-mf if s == 0 else 1.0)
    eye = np.eye(4 * Ls).reshape(Ls, 4, Ls, 4)
    B = b5 * eye + c5 * S
    A = (4.0 - M5) * B + eye - S
    return A, B


def _block_apply(M, psi, dagger=False):
    """(M psi) on a (Ls, V, 4, 3) field, M an (Ls, 4, Ls, 4) real block (M^T for dagger)."""
    if dagger:
        M = np.transpose(M, (2, 3, 0, 1))
    return np.einsum("satb,tvbc->svac", M, _c(psi))


def _hop5(L, bc, U, psi, dagger=False, out_parity=-1):
    return np.stack([hop(L, bc, U, p, dagger=dagger, out_parity=out_parity) for p in _c(psi)])


def mobius(L, bc, Ls, M5, mf, b5, c5, U, psi, dagger=False):
    """D_M psi = A psi - 1/2 H B psi (adjoint: A^T psi - 1/2 B^T H^dag psi) on (Ls, V, 4, 3)."""
    A, B = mobius_blocks(Ls, M5, mf, b5, c5)
    if not dagger:
        return _block_apply(A, psi) - 0.5 * _hop5(L, bc, U, _block_apply(B, psi))
    return _block_apply(A, psi, True) - 0.5 * _block_apply(B, _hop5(L, bc, U, psi, dagger=True), True)


def _block_inv(M):
    n = M.shape[0] * M.shape[1]
    return np.linalg.inv(M.reshape(n, n)).reshape(M.shape)


def mobius_mhat(L, bc, Ls, M5, mf, b5, c5, U, psi_even, dagger=False):
    """Even-odd operator of the Mobius matrix in the variable x' = B x: D B^-1 = A B^-1 - 1/2 H
    has the form of Eq. (2) with the site-local block A B^-1, whose inverse is W = B A^-1, and
      Mhat = 1 - 1/4 W H_eo W H_oe,   Mhat^dag = 1 - 1/4 H^dag_eo W^T H^dag_oe W^T
    (the Schur complement of D B^-1 on the even sites, times the inverse of its even block).
    Returns the even sites (odd sites zero)."""
    A, B = mobius_blocks(Ls, M5, mf, b5, c5)
    W = np.einsum("satb,tbuc->sauc", B, _block_inv(A))
    par = parity(L)
    pe = _c(psi_even).copy()
    pe[:, par == 1] = 0
    if not dagger:
        t = _block_apply(W, _hop5(L, bc, U, pe, out_parity=1))
        out = pe - 0.25 * _block_apply(W, _hop5(L, bc, U, t, out_parity=0))
    else:
        t = _hop5(L, bc, U, _block_apply(W, pe, True), dagger=True, out_parity=1)
        out = pe - 0.25 * _hop5(L, bc, U, _block_apply(W, t, True), dagger=True, out_parity=0)
    out[:, par == 1] = 0
    return out


def mobius_block(Ls, M5, mf, b5, c5, which, psi, dagger=False):
    """A, B, B^-1 or W = B A^-1 (which = "A", "B", "Binv", "W") applied to a (Ls, V, 4, 3) field."""
    A, B = mobius_blocks(Ls, M5, mf, b5, c5)
    M = {"A": A, "B": B, "Binv": _block_inv(B) if which == "Binv" else None,
         "W": np.einsum("satb,tbuc->sauc", B, _block_inv(A)) if which == "W" else None}[which]
    return _block_apply(M, psi, dagger)


def mobius_solve(L, bc, Ls, M5, mf, b5, c5, U, b, tol=1e-12, maxiter=20000):
    """Solve D_M x = b (Mobius, or Eq. (2) at b5 = 1, c5 = 0) through the even-odd system of
    D B^-1 in x' = B x: bhat = W (b_e + 1/2 H_eo W b_o), CG (Hestenes-Stiefel) on
    Mhat^dag Mhat x'_e = Mhat^dag bhat, x'_o = W (b_o + 1/2 H_oe x'_e), x = B^-1 x'.
    Returns (x, CG iterations, |b - D x| / |b|)."""
    par = parity(L)
    b = _c(b)
    be, bo = b.copy(), b.copy()
    be[:, par == 1] = 0
    bo[:, par == 0] = 0
    W = lambda v, dag=False: mobius_block(Ls, M5, mf, b5, c5, "W", v, dag)
    t = W(bo)
    t[:, par == 0] = 0
    bhat = W(be + 0.5 * _hop5(L, bc, U, t, out_parity=0))
    bhat[:, par == 1] = 0
    mh = lambda v, dag=False: mobius_mhat(L, bc, Ls, M5, mf, b5, c5, U, v, dagger=dag)
    rhs = mh(bhat, True)
    x = np.zeros_like(b)
    r = rhs.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    stop = (tol * np.linalg.norm(rhs)) ** 2
    it = 0
    while rr > stop and it < maxiter:
        q = mh(mh(p), True)
        alpha = rr / np.vdot(p, q).real
        x += alpha * p
        r -= alpha * q
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    t = x.copy()
    xo = W(bo + 0.5 * _hop5(L, bc, U, t, out_parity=1))
    xo[:, par == 0] = 0
    xp = x + xo
    xs = mobius_block(Ls, M5, mf, b5, c5, "Binv", xp)
    res = np.linalg.norm(b - mobius(L, bc, Ls, M5, mf, b5, c5, U, xs)) / np.linalg.norm(b)
    return xs, it, res

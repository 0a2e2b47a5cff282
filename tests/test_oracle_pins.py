"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the mathematics.

Nothing here compares the oracle with itself: each check uses a closed form, an
invariant, a special case that reduces to a library routine (dense numpy
algebra), or brute force on a tiny lattice.  The operators are those of
Kanamori & Matsufuru (arXiv:1712.01505): Eq. (1) (Wilson), Eq. (2)
(domain-wall), BiCGStab and CG of Sec. II C.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs

BC_T = (1, 1, 1, -1)  # periodic space, antiperiodic time


# ----------------------------------------------------------------------------- helpers
def dense(apply, shape, mask=None):
    """Dense matrix of a linear map on complex arrays of `shape` (columns = images of unit vectors)."""
    n = int(np.prod(shape))
    idx = np.arange(n) if mask is None else np.flatnonzero(mask)
    cols = []
    for j in idx:
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        cols.append(apply(e.reshape(shape)).reshape(-1)[idx])
    return np.array(cols).T


def match_spectra(a, b):
    """Largest distance in the optimal one-to-one matching of two eigenvalue multisets."""
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


def momenta(L, bc):
    """All lattice momenta p_mu = (2 pi n + (pi if antiperiodic)) / L_mu, shape (V, 4)."""
    axes = [(2 * np.pi * np.arange(l) + (np.pi if b < 0 else 0.0)) / l for l, b in zip(L, bc)]
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in grid], axis=-1)


def field_grid(a, L):
    """View a (V, ...) canonical field as (Lt, Lz, Ly, Lx, ...)."""
    Lx, Ly, Lz, Lt = L
    return a.reshape((Lt, Lz, Ly, Lx) + a.shape[1:])


def shift_fwd(a, L, mu):
    """b(x) = a(x + mu_hat) (periodic wrap; no boundary factor) for a canonical (V, ...) array."""
    axis = 3 - mu
    return np.roll(field_grid(a, L), -1, axis=axis).reshape(a.shape)


def gamma5_apply(psi):
    g5 = np.diag(ora.gamma(4))
    return psi * g5[:, None]


def vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


# ----------------------------------------------------------------------------- Dirac algebra
def test_clifford_algebra_and_gamma5():
    """gamma_mu Hermitian, {gamma_mu, gamma_nu} = 2 delta, gamma_5 = g1 g2 g3 g4 anticommutes."""
    g = [ora.gamma(k) for k in range(5)]
    I4 = np.eye(4)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * I4 * (m == n), atol=1e-15)
        assert np.allclose(g[4] @ g[m] + g[m] @ g[4], 0, atol=1e-15)
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    assert np.allclose(g[4] @ g[4], I4, atol=1e-15)


# ----------------------------------------------------------------------------- Wilson, Eq. (1)
def test_wilson_free_spectrum_closed_form():
    """U = 1: spectrum of M = 1 - kappa H is {1 - 2k sum cos p +- 2ik |sin p|}, each 6-fold."""
    L, kappa = (4, 2, 2, 6), 0.11
    V = ora.volume(L)
    U = inputs.unit_gauge(L)
    Md = dense(lambda v: ora.wilson(L, BC_T, kappa, U, v), (V, 4, 3))
    ev = np.linalg.eigvals(Md)
    p = momenta(L, BC_T)
    c = 1 - 2 * kappa * np.cos(p).sum(1)
    s = 2 * kappa * np.sqrt((np.sin(p) ** 2).sum(1))
    closed = np.concatenate([np.repeat(c + 1j * s, 6), np.repeat(c - 1j * s, 6)])
    assert match_spectra(ev, closed) < 1e-10


def test_wilson_forward_projector_is_one_minus_gamma():
    """Eq. (1): the forward hop from x to x+mu carries (1 - gamma_mu), the backward one (1 + gamma_mu).

    A unit spinor at site y that is a +1 eigenvector of gamma_mu is annihilated by
    (1 - gamma_mu), so it must not reach y - mu (whose forward hop reads y), while the
    backward hop of y + mu reads it with (1 + gamma_mu) = 2.
    """
    L = (4, 4, 4, 4)
    V = ora.volume(L)
    U = inputs.unit_gauge(L)
    y = 1 + 4 * (1 + 4 * (1 + 4 * 1))  # site (1,1,1,1)
    for mu in range(4):
        w, vec = np.linalg.eigh(ora.gamma(mu))
        u = vec[:, np.argmax(w)]  # gamma_mu u = +u
        psi = np.zeros((V, 4, 3), dtype=np.complex128)
        psi[y, :, 0] = u
        out = ora.hop((4, 4, 4, 4), (1, 1, 1, 1), U, psi)
        step = [1, 4, 16, 64][mu]
        assert np.abs(out[y - step]).max() < 1e-15
        assert np.allclose(out[y + step, :, 0], 2 * u, atol=1e-15)


def test_wilson_gauge_covariance():
    """D[U'](Omega psi) = Omega D[U] psi with U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag."""
    L = (4, 2, 4, 6)
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.5, 11)
    Om = inputs.random_gauge_transform(V, 12)
    psi = inputs.gaussian_source((V, 4, 3), 13)
    Up = np.empty_like(U)
    for mu in range(4):
        Up[mu] = Om @ U[mu] @ np.conj(np.swapaxes(shift_fwd(Om, L, mu), -1, -2))
    om_psi = np.einsum("xab,xsb->xsa", Om, psi)
    for dag in (False, True):
        lhs = ora.wilson(L, BC_T, 0.13, Up, om_psi, dagger=dag)
        rhs = np.einsum("xab,xsb->xsa", Om, ora.wilson(L, BC_T, 0.13, U, psi, dagger=dag))
        assert np.abs(lhs - rhs).max() < 1e-13


def test_wilson_gamma5_hermiticity_and_adjoint():
    """gamma5 M gamma5 = M^dag (from Eq. (1) and gamma Hermitian); <chi, M^dag psi> = <M chi, psi>."""
    L = (4, 4, 2, 4)
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.7, 21)
    chi = inputs.gaussian_source((V, 4, 3), 22)
    psi = inputs.gaussian_source((V, 4, 3), 23)
    k = 0.124
    Mdag_psi = ora.wilson(L, BC_T, k, U, psi, dagger=True)
    g5Mg5 = gamma5_apply(ora.wilson(L, BC_T, k, U, gamma5_apply(psi)))
    assert np.abs(Mdag_psi - g5Mg5).max() < 1e-13
    a = vdot(chi, Mdag_psi)
    b = vdot(ora.wilson(L, BC_T, k, U, chi), psi)
    assert abs(a - b) < 1e-11 * abs(a)


def test_hop_sites_matches_full_hop():
    """The sampled-site evaluation used at large volumes is the same map as the full one."""
    L = (4, 4, 2, 6)
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.3, 31)
    psi = inputs.gaussian_source((V, 4, 3), 32)
    sites = np.array([0, 5, 17, V - 1, V // 2])
    full = ora.hop(L, BC_T, U, psi)
    part = ora.hop_sites(L, BC_T, U, psi, sites)
    assert np.array_equal(full[sites], part)


def test_wilson_schur_complement_equals_dense_blocks():
    """Mhat = M_ee - M_eo M_oo^-1 M_oe, computed from dense blocks of the full M."""
    L = (2, 2, 2, 4)
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.5, 41)
    k = 0.12
    par = ora.parity(L)
    Md = dense(lambda v: ora.wilson(L, BC_T, k, U, v), (V, 4, 3))
    ev = np.repeat(par == 0, 12)
    od = ~ev
    S = Md[np.ix_(ev, ev)] - Md[np.ix_(ev, od)] @ np.linalg.solve(Md[np.ix_(od, od)], Md[np.ix_(od, ev)])
    for dag in (False, True):
        Mh = dense(lambda v: ora.wilson_mhat(L, BC_T, k, U, v, dagger=dag), (V, 4, 3), mask=ev)
        ref = S.conj().T if dag else S
        assert np.abs(Mh - ref).max() < 1e-14


@pytest.mark.parametrize("dagger", [False, True])
def test_wilson_solve_brute_force(dagger):
    """Even-odd BiCGStab + reconstruction equals numpy.linalg.solve on the dense full matrix."""
    L = (2, 2, 2, 4)
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.5, 51)
    b = inputs.gaussian_source((V, 4, 3), 52)
    k = 0.12
    Md = dense(lambda v: ora.wilson(L, BC_T, k, U, v, dagger=dagger), (V, 4, 3))
    x_np = np.linalg.solve(Md, b.reshape(-1)).reshape(V, 4, 3)
    x, it, res = ora.wilson_solve(L, BC_T, k, U, b, tol=1e-12, dagger=dagger)
    assert it > 0 and res <= 1e-12
    assert np.linalg.norm(x - x_np) <= 1e-10 * np.linalg.norm(x_np)


# ----------------------------------------------------------------------------- domain wall, Eq. (2)
DW_M5, DW_MF = 1.8, 0.02


def test_dw_free_spectrum_momentum_space():
    """U = 1: D_DW is block diagonal in momentum; its spectrum is the union over p of the
    4Ls x 4Ls matrices of Eq. (2) with D_W(p) = -M5 + sum(1 - cos p) + i sum gamma sin p."""
    L, Ls = (2, 2, 2, 4), 4
    V = ora.volume(L)
    U = inputs.unit_gauge(L)
    Dd = dense(lambda v: ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, v), (Ls, V, 4, 3))
    ev = np.linalg.eigvals(Dd)
    g = [ora.gamma(k) for k in range(5)]
    Pp, Pm = 0.5 * (np.eye(4) + g[4]), 0.5 * (np.eye(4) - g[4])
    closed = []
    for p in momenta(L, BC_T):
        Dw = (-DW_M5 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
        B = np.zeros((4 * Ls, 4 * Ls), dtype=np.complex128)
        for s in range(Ls):
            B[4 * s:4 * s + 4, 4 * s:4 * s + 4] = Dw + np.eye(4)
            if s + 1 < Ls:
                B[4 * s:4 * s + 4, 4 * (s + 1):4 * (s + 2)] = -Pm
            if s > 0:
                B[4 * s:4 * s + 4, 4 * (s - 1):4 * s] = -Pp
        B[0:4, 4 * (Ls - 1):] += DW_MF * Pp
        B[4 * (Ls - 1):, 0:4] += DW_MF * Pm
        closed.append(np.repeat(np.linalg.eigvals(B), 3))
    assert match_spectra(ev, np.concatenate(closed)) < 1e-9


def test_dw_gamma5_r5_hermiticity_and_adjoint():
    """(gamma5 R5) D_DW (gamma5 R5) = D_DW^dag, R5: s -> Ls-1-s; and <chi, D^dag psi> = <D chi, psi>."""
    L, Ls = (2, 4, 2, 4), 6
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.4, 61)
    chi = inputs.gaussian_source((Ls, V, 4, 3), 62)
    psi = inputs.gaussian_source((Ls, V, 4, 3), 63)

    def G(v):
        return gamma5_apply(v[::-1].reshape(Ls * V, 4, 3)).reshape(Ls, V, 4, 3)

    Ddag = ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, psi, dagger=True)
    assert np.abs(Ddag - G(ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, G(psi)))).max() < 1e-13
    a = vdot(chi, Ddag)
    b = vdot(ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, chi), psi)
    assert abs(a - b) < 1e-11 * abs(a)


def test_dw_gauge_covariance():
    L, Ls = (2, 4, 2, 4), 4
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.4, 71)
    Om = inputs.random_gauge_transform(V, 72)
    psi = inputs.gaussian_source((Ls, V, 4, 3), 73)
    Up = np.empty_like(U)
    for mu in range(4):
        Up[mu] = Om @ U[mu] @ np.conj(np.swapaxes(shift_fwd(Om, L, mu), -1, -2))
    rot = lambda v: np.einsum("xab,sxqb->sxqa", Om, v)
    lhs = ora.dw(L, BC_T, Ls, DW_M5, DW_MF, Up, rot(psi))
    rhs = rot(ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, psi))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_dw_block_inverse_closed_form():
    """The site-local block of Eq. (2) restricted to chirality +- is a I - (twisted shift) with
    a = 5 - M5 and wrap factor -m; its inverse has the closed form
    (A_+^-1)_{s s'} = a^(-1-k) (1 if s >= s' else -m) / (1 + m a^-Ls), k = (s - s') mod Ls,
    and A_-^-1 is its transpose.  The oracle inverts the block by elimination."""
    Ls, V = 8, 1
    a = 5 - DW_M5
    Ainv_plus = np.empty((Ls, Ls))
    for s in range(Ls):
        for sp in range(Ls):
            k = (s - sp) % Ls
            Ainv_plus[s, sp] = a ** (-1 - k) * (1.0 if s >= sp else -DW_MF) / (1 + DW_MF * a ** (-Ls))
    Ainv = dense(lambda v: ora.dw_ainv(Ls, V, DW_M5, DW_MF, v), (Ls, V, 4, 3))
    Ainv = Ainv.reshape(Ls, 4, 3, Ls, 4, 3)
    for sp in range(4):  # gamma_5 = diag(1,1,-1,-1): spins 0,1 are P_+, 2,3 are P_-
        blk = Ainv[:, sp, 0, :, sp, 0]
        ref = Ainv_plus if sp < 2 else Ainv_plus.T
        assert np.abs(blk - ref).max() < 1e-15
    # and it really inverts the block
    psi = inputs.gaussian_source((Ls, 3, 4, 3), 81)
    back = ora.dw_block(Ls, 3, DW_M5, DW_MF, ora.dw_ainv(Ls, 3, DW_M5, DW_MF, psi))
    assert np.abs(back - psi).max() < 1e-14


def test_dw_schur_complement_equals_dense_blocks():
    """Mhat = D_ee^-1 (D_ee - D_eo D_oo^-1 D_oe) from dense blocks of the full D_DW."""
    L, Ls = (2, 2, 2, 4), 4
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.4, 91)
    par = ora.parity(L)
    Dd = dense(lambda v: ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, v), (Ls, V, 4, 3))
    ev = np.tile(np.repeat(par == 0, 12), Ls)
    od = ~ev
    Dee, Deo, Doe, Doo = (Dd[np.ix_(r, c)] for r, c in ((ev, ev), (ev, od), (od, ev), (od, od)))
    S = np.linalg.solve(Dee, Dee - Deo @ np.linalg.solve(Doo, Doe))
    for dag in (False, True):
        Mh = dense(lambda v: ora.dw_mhat(L, BC_T, Ls, DW_M5, DW_MF, U, v, dagger=dag),
                   (Ls, V, 4, 3), mask=ev)
        ref = S.conj().T if dag else S
        assert np.abs(Mh - ref).max() < 1e-13


def test_dw_solve_brute_force():
    L, Ls = (2, 2, 2, 4), 4
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.4, 101)
    b = inputs.gaussian_source((Ls, V, 4, 3), 102)
    Dd = dense(lambda v: ora.dw(L, BC_T, Ls, DW_M5, DW_MF, U, v), (Ls, V, 4, 3))
    x_np = np.linalg.solve(Dd, b.reshape(-1)).reshape(b.shape)
    x, it, res = ora.dw_solve(L, BC_T, Ls, DW_M5, DW_MF, U, b, tol=1e-11)
    assert it > 0 and res <= 1e-11
    assert np.linalg.norm(x - x_np) <= 1e-8 * np.linalg.norm(x_np)


# ----------------------------------------------------------------------------- force
def _action(L, k, U, phi):
    S, _, _ = ora.wilson_action(L, BC_T, k, U, phi, tol=1e-14)
    return S


def _fd_check(L, k, U, phi, comps, h=1e-5, rtol=1e-6):
    S0, eta, X = ora.wilson_action(L, BC_T, k, U, phi, tol=1e-14)
    g = ora.wilson_force(L, BC_T, k, X, eta)
    scale = np.sqrt(np.mean(g ** 2))
    for (mu, x, a, b, ri) in comps:
        d = np.zeros_like(U)
        d[mu, x, a, b] = h * (1.0 if ri == 0 else 1j)
        fd = (_action(L, k, U + d, phi) - _action(L, k, U - d, phi)) / (2 * h)
        assert abs(fd - g[mu, x, a, b, ri]) <= rtol * max(abs(fd), scale), (mu, x, a, b, ri)


def test_force_finite_differences_all_components_small():
    """dS/dU (18 independent reals per link) against central differences of S, every component."""
    L, k = (2, 2, 2, 4), 0.12
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.5, 111)
    phi = inputs.gaussian_source((V, 4, 3), 112)
    comps = [(mu, x, a, b, ri) for mu in range(4) for x in range(V) for a in range(3)
             for b in range(3) for ri in range(2)]
    _fd_check(L, k, U, phi, comps)


def test_force_finite_differences_sampled_4x4x4x4():
    """Same on a lattice where x+mu and x-mu differ in every direction (sampled components)."""
    L, k = (4, 4, 4, 4), 0.12
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.3, 121)
    phi = inputs.gaussian_source((V, 4, 3), 122)
    rng = np.random.default_rng(123)
    comps = [(mu, int(rng.integers(V)), int(rng.integers(3)), int(rng.integers(3)), int(rng.integers(2)))
             for mu in range(4) for _ in range(8)]
    _fd_check(L, k, U, phi, comps)


# ----------------------------------------------------------------------------- inputs
def test_generator_su3_and_smoothness():
    """Links are SU(3) (unitary, det 1) and the mean plaquette -> 1 as eps -> 0."""
    L = (4, 4, 4, 4)
    means = []
    for eps, lo in ((0.05, 0.98), (0.3, 0.5)):
        U = inputs.gauge_field(L, eps, 5)
        I3 = np.eye(3)
        assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I3).max() < 1e-14
        assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
        plaq = []
        for mu in range(4):
            for nu in range(mu + 1, 4):
                P = U[mu] @ shift_fwd(U[nu], L, mu) @ np.conj(np.swapaxes(shift_fwd(U[mu], L, nu), -1, -2)) \
                    @ np.conj(np.swapaxes(U[nu], -1, -2))
                plaq.append(np.trace(P, axis1=-2, axis2=-1).real.mean() / 3)
        assert lo < np.mean(plaq) <= 1.0
        means.append(np.mean(plaq))
    assert means[0] > means[1]
    # reproducible from the seed
    assert np.array_equal(inputs.gauge_field((2, 2, 2, 2), 0.2, 7), inputs.gauge_field((2, 2, 2, 2), 0.2, 7))


def test_spectra_explain_the_choice_of_solver():
    """Sec. II C: BiCGStab is used for Wilson and CG on D^dag D for domain-wall because the
    domain-wall spectrum reaches into the left half of the complex plane.  Dense spectra on 2^4
    (Ls = 4, M5 = 1.8, mf = 0.02) of the benchmark-like smoothed fields: every eigenvalue of the
    Wilson matrix at kappa = 0.125 has a positive real part, some of the domain-wall ones do not."""
    L = (2, 2, 2, 2)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 3)
    n4 = V * 12
    W = np.empty((n4, n4), dtype=complex)
    for j in range(n4):
        e = np.zeros(n4, dtype=complex)
        e[j] = 1.0
        W[:, j] = ora.wilson(L, BC_T, 0.125, U, e.reshape(V, 4, 3)).reshape(n4)
    ew = np.linalg.eigvals(W)
    Ls = 4
    n5 = Ls * n4
    D = np.empty((n5, n5), dtype=complex)
    for j in range(n5):
        e = np.zeros(n5, dtype=complex)
        e[j] = 1.0
        D[:, j] = ora.dw(L, BC_T, Ls, 1.8, 0.02, U, e.reshape(Ls, V, 4, 3)).reshape(n5)
    ed = np.linalg.eigvals(D)
    assert ew.real.min() > 0
    assert ed.real.min() < 0 < ed.real.max()


def test_oracle_results_do_not_depend_on_the_thread_count():
    """The benchmark times the oracle on one thread and on all; each output site is computed
    independently, so the results are identical."""
    L = (4, 4, 2, 6)
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.3, 71)
    psi = inputs.gaussian_source((V, 4, 3), 72)
    n = ora.num_threads()
    try:
        ora.set_num_threads(1)
        a = ora.wilson(L, BC_T, 0.12, U, psi)
        ora.set_num_threads(max(n, 2))
        b = ora.wilson(L, BC_T, 0.12, U, psi)
    finally:
        ora.set_num_threads(n)
    assert np.array_equal(a, b)


def test_action_gauge_invariance_and_force_covariance():
    """S[U', Omega phi] = S[U, phi] with U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag, and the link
    gradient G = dS/dRe U + i dS/dIm U transforms as G'_mu(x) = Omega(x) G_mu(x) Omega(x+mu)^dag
    (S is invariant, so dS = Re tr(G^dag dU) must be too)."""
    L, k = (4, 2, 2, 4), 0.12
    V = ora.volume(L)
    U = inputs.gauge_field(L, 0.4, 121)
    Om = inputs.random_gauge_transform(V, 122)
    phi = inputs.gaussian_source((V, 4, 3), 123)

    def transform(M):  # Omega(x) M_mu(x) Omega(x+mu)^dag for a (4, V, 3, 3) array
        out = np.empty_like(M)
        for mu in range(4):
            out[mu] = Om @ M[mu] @ np.conj(np.swapaxes(shift_fwd(Om, L, mu), -1, -2))
        return out

    S0, eta, X = ora.wilson_action(L, BC_T, k, U, phi, tol=1e-14)
    S1, eta1, X1 = ora.wilson_action(L, BC_T, k, transform(U), np.einsum("xab,xsb->xsa", Om, phi), tol=1e-14)
    assert abs(S1 - S0) <= 1e-11 * S0
    g0 = ora.wilson_force(L, BC_T, k, X, eta)
    g1 = ora.wilson_force(L, BC_T, k, X1, eta1)
    G0 = g0[..., 0] + 1j * g0[..., 1]
    G1 = g1[..., 0] + 1j * g1[..., 1]
    assert np.abs(G1 - transform(G0)).max() <= 1e-10 * np.abs(G0).max()

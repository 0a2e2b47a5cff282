"""Pins of the oracle's molecular-dynamics pieces (even-odd pseudofermion action, its force
projected onto su(3), exp(eps P) U, leapfrog) against definitions that do not go through them:
dense linear algebra, finite differences along su(3) directions, group properties, and the
leapfrog's error order and time reversibility."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs

BC = (1, 1, 1, -1)


def _herm_traceless(rng):
    a = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    h = 0.5 * (a + a.conj().T)
    return h - np.trace(h) / 3 * np.eye(3)


def test_eo_action_equals_dense_schur_complement():
    L, kappa = (2, 2, 2, 4), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.4, 3)
    phi = inputs.gaussian_source((V, 4, 3), 4)
    par = ora.parity(L)
    even = np.flatnonzero(par == 0)
    n = len(even) * 12
    # Mhat column by column from unit vectors on the even sites
    M = np.empty((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros((V, 4, 3), dtype=complex)
        e[even[j // 12]].reshape(12)[j % 12] = 1.0
        M[:, j] = ora.wilson_mhat(L, BC, kappa, U, e)[even].reshape(n)
    pe = phi[even].reshape(n)
    s_dense = np.vdot(pe, np.linalg.solve(M.conj().T @ M, pe)).real
    s, X, Y = ora.wilson_eo_action(L, BC, kappa, U, phi)
    assert abs(s - s_dense) <= 1e-11 * s_dense
    # X = (Mhat^dag Mhat)^-1 phi_e and Y = Mhat X on the even sites, zero on the odd ones
    assert np.allclose(X[even].reshape(n), np.linalg.solve(M.conj().T @ M, pe), atol=1e-11)
    assert np.allclose(Y[even].reshape(n), M @ X[even].reshape(n), atol=1e-11)
    assert not X[par == 1].any() and not Y[par == 1].any()


@pytest.mark.parametrize("L", [(2, 2, 2, 4), (4, 2, 2, 2)])
def test_projected_eo_force_matches_finite_differences(L):
    kappa = 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.4, 5)
    phi = inputs.gaussian_source((V, 4, 3), 6)
    _, X, Y = ora.wilson_eo_action(L, BC, kappa, U, phi)
    F = ora.su3_project(U, ora.wilson_eo_force(L, BC, kappa, U, X, Y))
    # su(3): anti-Hermitian and traceless
    assert np.allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-13)
    assert np.allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-13)
    from scipy.linalg import expm

    rng = np.random.default_rng(7)
    eps = 1e-4
    for _ in range(6):
        mu, x = int(rng.integers(4)), int(rng.integers(V))
        T = _herm_traceless(rng)
        sp = []
        for sgn in (1, -1):
            U2 = U.copy()
            U2[mu, x] = expm(1j * sgn * eps * T) @ U[mu, x]
            sp.append(ora.wilson_eo_action(L, BC, kappa, U2, phi)[0])
        fd = (sp[0] - sp[1]) / (2 * eps)
        an = np.trace(1j * T @ F[mu, x])
        assert abs(an.imag) < 1e-12
        assert abs(fd - an.real) <= 1e-6 * max(abs(fd), 1e-3), (mu, x, fd, an)


def test_link_update_is_a_group_action():
    rng_shape = (64,)
    P = inputs.su3_momenta(rng_shape, 8)
    U = inputs.gauge_field((2, 2, 2, 2), 0.5, 9).reshape(-1, 3, 3)[:64]
    U1 = ora.link_update(U, P, 0.3)
    eye = np.broadcast_to(np.eye(3), U1.shape)
    assert np.allclose(U1 @ np.conj(np.swapaxes(U1, -1, -2)), eye, atol=1e-13)
    assert np.allclose(np.linalg.det(U1), 1.0, atol=1e-13)
    assert np.allclose(ora.link_update(U1, P, -0.3), U, atol=1e-13)
    # first order: U + eps P U
    d = 1e-6
    assert np.allclose((ora.link_update(U, P, d) - U) / d, P @ U, atol=1e-5)


def _md_case():
    L, kappa = (2, 2, 2, 4), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 10)
    P = inputs.su3_momenta((4, V), 11)
    phi = inputs.gaussian_source((V, 4, 3), 12)
    return L, kappa, U, P, phi


def test_leapfrog_energy_error_is_second_order():
    L, kappa, U, P, phi = _md_case()
    tau = 0.2
    dh = []
    for n in (2, 4, 8):
        _, _, h0, h1 = ora.leapfrog(L, BC, kappa, U, P, phi, tau / n, n)
        dh.append(abs(h1 - h0))
    assert dh[0] > dh[1] > dh[2] > 0
    for a, b in zip(dh, dh[1:]):
        assert 3.0 < a / b < 5.3, dh


def test_leapfrog_is_reversible():
    L, kappa, U, P, phi = _md_case()
    U1, P1, h0, h1 = ora.leapfrog(L, BC, kappa, U, P, phi, 0.05, 4)
    U2, P2, h2, h3 = ora.leapfrog(L, BC, kappa, U1, -P1, phi, 0.05, 4)
    assert np.allclose(U2, U, atol=1e-10)
    assert np.allclose(-P2, P, atol=1e-10)
    assert abs(h3 - h0) < 1e-9

"""Pins of the oracle's Mobius domain-wall operator D = D_W B + 1 - S (B = b5 + c5 S):
Eq. (2) at b5 = 1, c5 = 0; the adjoint and gamma5 R5 hermiticity (c5 = 0); the free spectrum in
momentum space; the induced 4D overlap operator (polar sign approximation), which fixes the order
of D_W and the s-hop; the even-odd operator against the dense Schur complement of D B^-1; the blocks; a dense solve."""
import numpy as np

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs
from tests.test_oracle_pins import match_spectra, momenta

BC = (1, 1, 1, -1)
M5, MF = 1.8, 0.02
B5_PIN, C5_PIN = 1.5, 0.5


def _dense(op, n):
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(op(e))
    return np.stack(cols, axis=1)


def test_b5_1_c5_0_is_the_shamir_operator_of_eq2():
    L, Ls = (4, 2, 2, 4), 6
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 1)
    psi = inputs.gaussian_source((Ls, V, 4, 3), 2)
    for dag in (False, True):
        a = ora.mobius(L, BC, Ls, M5, MF, 1.0, 0.0, U, psi, dagger=dag)
        b = ora.dw(L, BC, Ls, M5, MF, U, psi, dagger=dag)
        assert np.allclose(a, b, atol=1e-13)
        am = ora.mobius_mhat(L, BC, Ls, M5, MF, 1.0, 0.0, U, psi, dagger=dag)
        par = ora.parity(L)
        pe = psi.copy()
        pe[:, par == 1] = 0
        bm = ora.dw_mhat(L, BC, Ls, M5, MF, U, pe, dagger=dag)
        assert np.allclose(am, bm, atol=1e-12)


def test_adjoint_and_gamma5_r5_hermiticity_at_c5_0():
    """D^dag is the conjugate transpose of D for any (b5, c5).  At c5 = 0 (B = b5 times the
    identity) (gamma5 R5) D (gamma5 R5) = D^dag, R5: s -> Ls-1-s.  With c5 != 0 that relation does
    not hold for D = D_W B + 1 - S, since D_W does not commute with the chiral projectors in S
    (the solver takes CG on the normal equations, which does not need it)."""
    L, Ls = (2, 2, 2, 4), 4
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 3)
    n = Ls * V * 12
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    G = np.zeros((Ls, V, 4, 3, Ls, V, 4, 3))
    for s in range(Ls):
        for v in range(V):
            for c in range(3):
                G[s, v, :, c, Ls - 1 - s, v, :, c] = g5
    G = G.reshape(n, n)
    for b5, c5 in ((1.5, 0.5), (1.7, 0.0)):
        D = _dense(lambda e: ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, e.reshape(Ls, V, 4, 3)).reshape(n), n)
        Dd = _dense(lambda e: ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, e.reshape(Ls, V, 4, 3),
                                         dagger=True).reshape(n), n)
        assert np.allclose(Dd, D.conj().T, atol=1e-13)
        herm = np.abs(G @ D @ G - D.conj().T).max()
        assert (herm < 1e-12) == (c5 == 0.0), (b5, c5, herm)


def test_free_spectrum_momentum_space():
    """U = 1: D is block diagonal in momentum.  For each p the 4Ls x 4Ls block is
    (b5 D_W(p) + 1) delta_{s,s'} + (c5 D_W(p) - 1) S_{s,s'}, with
    D_W(p) = -M5 + sum(1 - cos p) + i sum gamma sin p and S the chiral hop in s
    (P- from s+1, P+ from s-1, -mf at the walls): D_W acts after the s-hop."""
    L, Ls, b5, c5 = (2, 2, 2, 4), 4, 1.5, 0.5
    V = int(np.prod(L))
    U = inputs.unit_gauge(L)
    n = Ls * V * 12
    D = _dense(lambda e: ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, e.reshape(Ls, V, 4, 3)).reshape(n), n)
    ev = np.linalg.eigvals(D)
    g = [ora.gamma(k) for k in range(5)]
    Pp, Pm = 0.5 * (np.eye(4) + g[4]), 0.5 * (np.eye(4) - g[4])
    S = np.zeros((4 * Ls, 4 * Ls), dtype=complex)
    for s in range(Ls):
        if s + 1 < Ls:
            S[4 * s:4 * s + 4, 4 * (s + 1):4 * (s + 2)] = Pm
        if s > 0:
            S[4 * s:4 * s + 4, 4 * (s - 1):4 * s] = Pp
    S[0:4, 4 * (Ls - 1):] = -MF * Pp
    S[4 * (Ls - 1):, 0:4] = -MF * Pm
    closed = []
    for p in momenta(L, BC):
        Dw = (-M5 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
        K = np.kron(np.eye(Ls), Dw)
        closed.append(np.repeat(np.linalg.eigvals(b5 * K + np.eye(4 * Ls) + (c5 * K - np.eye(4 * Ls)) @ S), 3))
    assert match_spectra(ev, np.concatenate(closed)) < 1e-9


def test_effective_4d_operator_is_the_polar_sign_approximation():
    """The 4D operator a Mobius domain-wall fermion induces on its wall modes is the overlap
    operator with the Ls-th polar approximation of the sign function:
      [P^-1 D(1)^-1 D(mf) P]_{00} = (1 + mf)/2 + (1 - mf)/2 gamma5 eps(H_M),
      H_M = gamma5 (b5 + c5) D_W (2 + (b5 - c5) D_W)^-1,
      eps(H) = ((1 + H)^Ls - (1 - H)^Ls) ((1 + H)^Ls + (1 - H)^Ls)^-1,
    D_W = 4 - M5 - H/2 the 4D Wilson operator, (P psi)_s = P- psi_s + P+ psi_{s+1} (cyclic in s)
    and D(1) the operator at mf = 1.  This fixes the order of D_W and the s-hop in D (D_W acting
    after it), which the free spectrum cannot tell apart."""
    L, Ls, b5, c5, mf = (2, 2, 2, 4), 4, 1.5, 0.5, 0.1
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 8)
    n4 = V * 12
    n = Ls * n4

    def D(m):
        return _dense(lambda e: ora.mobius(L, BC, Ls, M5, m, b5, c5, U, e.reshape(Ls, V, 4, 3)).reshape(n), n)

    I = np.eye(n4)
    Dw = (4.0 - M5) * I - 0.5 * _dense(lambda e: ora.hop(L, BC, U, e.reshape(V, 4, 3)).reshape(n4), n4)
    g5 = np.kron(np.eye(V), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    Pp, Pm = 0.5 * (I + g5), 0.5 * (I - g5)
    HM = g5 @ ((b5 + c5) * Dw) @ np.linalg.inv(2.0 * I + (b5 - c5) * Dw)
    up, dn = np.linalg.matrix_power(I + HM, Ls), np.linalg.matrix_power(I - HM, Ls)
    sign = (up - dn) @ np.linalg.inv(up + dn)
    P = np.zeros((n, n))
    for s in range(Ls):
        t = (s + 1) % Ls
        P[s * n4:(s + 1) * n4, s * n4:(s + 1) * n4] += Pm
        P[s * n4:(s + 1) * n4, t * n4:(t + 1) * n4] += Pp
    Q = np.linalg.solve(P, np.linalg.solve(D(1.0), D(mf) @ P))
    want = 0.5 * (1 + mf) * I + 0.5 * (1 - mf) * g5 @ sign
    assert np.abs(Q[:n4, :n4] - want).max() < 1e-12


def test_even_odd_operator_is_the_schur_complement():
    """Mhat is the Schur complement of D' = D B^-1 on the even sites, times (D'_ee)^-1; and
    B_e^-1 Mhat B_e is the Schur complement of D itself, times (D_ee)^-1 (the two are similar)."""
    L, Ls, b5, c5 = (2, 2, 2, 4), 4, 1.5, 0.5
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 4)
    par = ora.parity(L)
    shape = (Ls, V, 4, 3)
    n = Ls * V * 12
    D = _dense(lambda e: ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, e.reshape(shape)).reshape(n), n)
    B = _dense(lambda e: ora.mobius_block(Ls, M5, MF, b5, c5, "B", e.reshape(shape)).reshape(n), n)
    mask = np.broadcast_to(par[None, :, None, None], shape).reshape(n)
    e, o = np.flatnonzero(mask == 0), np.flatnonzero(mask == 1)

    def schur(M):
        Mee, Meo, Moe, Moo = M[np.ix_(e, e)], M[np.ix_(e, o)], M[np.ix_(o, e)], M[np.ix_(o, o)]
        return np.linalg.solve(Mee, Mee - Meo @ np.linalg.solve(Moo, Moe))

    mhat = schur(D @ np.linalg.inv(B))
    Be = B[np.ix_(e, e)]
    assert np.abs(np.linalg.solve(Be, mhat @ Be) - schur(D)).max() < 1e-11
    psi = inputs.gaussian_source(shape, 5)
    for dag in (False, True):
        got = ora.mobius_mhat(L, BC, Ls, M5, MF, b5, c5, U, psi, dagger=dag).reshape(n)[e]
        want = (mhat.conj().T if dag else mhat) @ psi.reshape(n)[e]
        assert np.allclose(got, want, atol=1e-12)


def test_blocks():
    """B^-1 B = 1, W A = B, and A, B are the site-local parts of D (D = A - 1/2 H B)."""
    L, Ls, b5, c5 = (2, 2, 2, 2), 6, 1.5, 0.5
    V = int(np.prod(L))
    psi = inputs.gaussian_source((Ls, V, 4, 3), 9)
    blk = lambda w, v, dag=False: ora.mobius_block(Ls, M5, MF, b5, c5, w, v, dag)
    for dag in (False, True):
        assert np.abs(blk("Binv", blk("B", psi, dag), dag) - psi).max() < 1e-13
    assert np.abs(blk("W", blk("A", psi)) - blk("B", psi)).max() < 1e-13
    zero = np.zeros((4, V, 3, 3), dtype=complex)  # H = 0 without links
    assert np.abs(ora.mobius(L, BC, Ls, M5, MF, b5, c5, zero, psi) - blk("A", psi)).max() < 1e-14


def test_dense_solve():
    L, Ls, b5, c5 = (2, 2, 2, 4), 4, 1.5, 0.5
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 6)
    shape = (Ls, V, 4, 3)
    n = Ls * V * 12
    D = _dense(lambda e: ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, e.reshape(shape)).reshape(n), n)
    b = inputs.gaussian_source(shape, 7).reshape(n)
    x = np.linalg.solve(D, b)
    assert np.linalg.norm(ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, x.reshape(shape)).reshape(n) - b) < 1e-11


def test_even_odd_solve_equals_the_dense_solution():
    """The oracle's even-odd CG solve (x' = B x, Schur system of D B^-1, reconstruction, B^-1)
    reproduces numpy.linalg.solve on the dense D, Mobius and Shamir."""
    L, Ls = (2, 2, 2, 4), 4
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 10)
    shape = (Ls, V, 4, 3)
    n = Ls * V * 12
    b = inputs.gaussian_source(shape, 11)
    for b5, c5 in ((B5_PIN, C5_PIN), (1.0, 0.0)):
        D = _dense(lambda e: ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, e.reshape(shape)).reshape(n), n)
        xd = np.linalg.solve(D, b.reshape(n)).reshape(shape)
        x, it, res = ora.mobius_solve(L, BC, Ls, M5, MF, b5, c5, U, b, tol=1e-13)
        assert res <= 1e-12 and it > 0
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)

"""GPU molecular-dynamics pieces against the oracle: the even-odd pseudofermion force
(qcd_force_eo), its su(3) projection (qcd_force_project), exp(eps P) U (qcd_link_update),
the momentum update and kinetic term, and whole leapfrog trajectories (energy error of
second order, time reversibility, agreement with the oracle's trajectory).

Tolerances: the link kernels are FP64 (1e-13 of the largest entry, rounding of a few
dozen operations); quantities behind a solve carry the solver's 1e-12 relative residual."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import hmc, inputs, qcd
from tests.gpu_util import device, max_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 2, 10)])
def test_force_eo_parity(L):
    device()
    kappa = 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.4, 21)
    X = inputs.gaussian_source((V, 4, 3), 22)
    Y = inputs.gaussian_source((V, 4, 3), 23)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(kappa)
    out = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=device())
    qcd.force_eo(g, f, to_dev(X), to_dev(Y), out)
    torch.cuda.synchronize()
    assert max_err(out, ora.wilson_eo_force(L, BC, kappa, U, X, Y)) < 1e-13


def test_force_project_parity():
    device()
    L = (4, 4, 2, 6)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.5, 24)
    dS = np.random.default_rng(25).standard_normal((4, V, 3, 3, 2))
    g = qcd.Gauge.load(to_dev(U), L, BC)
    F = torch.empty((4, V, 3, 3), dtype=torch.complex128, device=device())
    qcd.force_project(g, to_dev(dS), F)
    torch.cuda.synchronize()
    ref = ora.su3_project(U, dS)
    assert max_err(F, ref) < 1e-13
    Fh = F.cpu().numpy()
    assert np.allclose(np.trace(Fh, axis1=-2, axis2=-1), 0, atol=1e-13)


def test_link_and_momentum_updates():
    device()
    n = 4 * 4 * 4 * 4 * 4
    U = inputs.gauge_field((4, 4, 4, 4), 0.5, 26)
    P = inputs.su3_momenta((4, 256), 27)
    for eps in (0.05, -0.7, 3.0):  # 3.0 needs several squarings
        Ud = to_dev(U)
        qcd.link_update(Ud, to_dev(P), eps)
        torch.cuda.synchronize()
        assert max_err(Ud, ora.link_update(U, P, eps)) < 1e-13
    Fm = inputs.su3_momenta((4, 256), 28)
    Pd = to_dev(P)
    qcd.mom_update(Pd, to_dev(Fm), -0.3)
    torch.cuda.synchronize()
    assert max_err(Pd, P - 0.3 * Fm) < 1e-15
    e = qcd.mom_energy(Pd)
    ref = ora.kinetic(P - 0.3 * Fm)
    assert abs(e - ref) <= 1e-12 * ref
    assert n == U.shape[0] * U.shape[1]


def test_action_and_force_match_the_oracle():
    device()
    L, kappa = (4, 4, 4, 4), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 29)
    phi = inputs.gaussian_source((V, 4, 3), 30)
    md = hmc.EOPseudofermionMD(L, kappa, to_dev(phi), tol=1e-12)
    F, S = md.force(to_dev(U))
    s_ref, X, Y = ora.wilson_eo_action(L, BC, kappa, U, phi)
    f_ref = ora.su3_project(U, ora.wilson_eo_force(L, BC, kappa, U, X, Y))
    assert abs(S - s_ref) <= 1e-10 * s_ref
    assert max_err(F, f_ref) < 1e-9


def _md_case(L=(4, 4, 4, 4)):
    kappa = 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 31)
    P = inputs.su3_momenta((4, V), 32)
    phi = inputs.gaussian_source((V, 4, 3), 33)
    return L, kappa, U, P, phi


def test_leapfrog_energy_error_is_second_order():
    device()
    L, kappa, U, P, phi = _md_case()
    md = hmc.EOPseudofermionMD(L, kappa, to_dev(phi), tol=1e-12)
    tau, dh = 0.2, []
    for n in (2, 4, 8):
        h0, h1 = md.leapfrog(to_dev(U), to_dev(P), tau / n, n)
        dh.append(abs(h1 - h0))
    for a, b in zip(dh, dh[1:]):
        assert 3.0 < a / b < 5.3, dh


def test_leapfrog_reversible_and_matches_the_oracle():
    device()
    L, kappa, U, P, phi = _md_case((2, 2, 2, 4))
    md = hmc.EOPseudofermionMD(L, kappa, to_dev(phi), tol=1e-12)
    Ud, Pd = to_dev(U), to_dev(P)
    h0, h1 = md.leapfrog(Ud, Pd, 0.05, 4)
    U1, P1, o0, o1 = ora.leapfrog(L, BC, kappa, U, P, phi, 0.05, 4)
    assert abs(h0 - o0) <= 1e-10 * abs(o0)
    assert abs((h1 - h0) - (o1 - o0)) <= 1e-8
    assert max_err(Ud, U1) < 1e-10 and max_err(Pd, P1) < 1e-8
    Pd.neg_()
    md.leapfrog(Ud, Pd, 0.05, 4)
    assert max_err(Ud, U) < 1e-9
    assert max_err(-Pd, P) < 1e-8


def test_eo_autograd_matches_the_oracle():
    """torch.autograd through the even-odd action: dS/dU is the oracle's even-odd force, dS/dphi is
    2 X on the even sites and 0 on the odd ones."""
    device()
    from paper_1712_01505_gb300.autograd import wilson_eo_action

    L, kappa = (6, 4, 4, 8), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 34)
    phi = inputs.gaussian_source((V, 4, 3), 35)
    Ut = to_dev(U).requires_grad_(True)
    pt = to_dev(phi).requires_grad_(True)
    S = wilson_eo_action(Ut, pt, kappa, L, BC, tol=1e-12)
    S.backward()
    s_ref, X, Y = ora.wilson_eo_action(L, BC, kappa, U, phi)
    assert abs(S.item() - s_ref) <= 1e-10 * s_ref
    g_ref = ora.wilson_eo_force(L, BC, kappa, U, X, Y)
    assert max_err(torch.view_as_real(Ut.grad), g_ref) < 1e-9
    assert max_err(pt.grad, 2 * X) < 1e-9
    assert not pt.grad.cpu().numpy()[ora.parity(L) == 1].any()

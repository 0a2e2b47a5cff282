"""GPU force kernel and the differentiable action S = phi^dag (M^dag M)^-1 phi (Wilson),
against the FP64 oracle's force formula, the oracle's gradient and central finite differences."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def test_force_kernel_parity_random_fields():
    """The outer-product kernel is bilinear in (X, eta): compare on random fields."""
    device()
    L = (6, 4, 4, 8)
    V = int(np.prod(L))
    X = inputs.gaussian_source((V, 4, 3), 81)
    eta = inputs.gaussian_source((V, 4, 3), 82)
    U = inputs.gauge_field(L, 0.3, 83)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.13)
    out = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=device())
    qcd.force(g, f, to_dev(X), to_dev(eta), out)
    torch.cuda.synchronize()
    assert max_err(out, ora.wilson_force(L, BC, 0.13, X, eta)) < 1e-13


def test_norm2_matches_numpy():
    device()
    L = (4, 4, 4, 4)
    V = int(np.prod(L))
    g = qcd.Gauge.load(to_dev(inputs.unit_gauge(L)), L, BC)
    psi = inputs.gaussian_source((3, V, 4, 3), 84)
    got = qcd.norm2(g, qcd.wilson(0.1), to_dev(psi), nrhs=3)
    want = [float(np.vdot(p, p).real) for p in psi]
    assert np.allclose(got, want, rtol=1e-14)
    assert np.allclose(qcd.norm2(g, qcd.wilson(0.1), psi, nrhs=3), want, rtol=1e-14)  # host buffer


@pytest.fixture(scope="module")
def config5():
    """16^4, eps = 0.3 links (seed 5), kappa = 0.12, Gaussian phi (seed 0)."""
    L, kappa = (16, 16, 16, 16), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 5)
    phi = inputs.gaussian_source((V, 4, 3), 0)
    return L, kappa, U, phi


def test_autograd_matches_oracle_gradient(config5):
    device()
    from paper_1712_01505_gb300.autograd import wilson_action

    L, kappa, U, phi = config5
    Ut = to_dev(U).requires_grad_(True)
    pt = to_dev(phi).requires_grad_(True)
    S = wilson_action(Ut, pt, kappa, L, BC, tol=1e-12, inner="f32")
    S.backward()
    S_o, eta_o, X_o = ora.wilson_action(L, BC, kappa, U, phi, tol=1e-12)
    assert abs(S.item() - S_o) <= 1e-10 * S_o
    g_o = ora.wilson_force(L, BC, kappa, X_o, eta_o)
    g = torch.view_as_real(Ut.grad).cpu().numpy()
    assert rel_err(g, g_o) < 1e-8
    assert rel_err(pt.grad, 2 * X_o) < 1e-8


# FD tolerance per step.  S = 2.08e6 here, one FP64 ulp of S is 4.6e-10, and at h = 1e-6 the
# numerator S+ - S- of a gradient component of rms size (3.2) is 6.4e-6 = 1.4e4 ulps: the FP64
# resolution of S itself caps the quotient at about 1e-4 per ulp of noise, and the two solves
# differ by ~10 ulps (measured worst deviation 1.1e-3).  At h = 1e-4 the quotient resolves the
# gradient to ~1e-5 (truncation O(h^2) is far below), so that step carries the tight bound;
# the oracle gradient (test above) is the 1e-8 pin.
FD_TOL = {1e-6: 5e-3, 1e-4: 1e-4}


@pytest.mark.parametrize("h", [1e-6, 1e-4])
def test_autograd_central_finite_differences(config5, h):
    """dS/dU on 64 random link components against (S(U + h e) - S(U - h e)) / 2h.

    Both perturbed solves start from the unperturbed solution and run the same fixed number
    of FP64 iterations (deterministic reductions), so their rounding errors largely cancel.
    """
    device()
    from paper_1712_01505_gb300.autograd import wilson_action

    L, kappa, U, phi = config5
    V = int(np.prod(L))
    Ut = to_dev(U).requires_grad_(True)
    S = wilson_action(Ut, to_dev(phi), kappa, L, BC, tol=1e-12, inner="f32")
    S.backward()
    g = torch.view_as_real(Ut.grad).cpu().numpy()
    f = qcd.wilson(kappa)
    phi_d = to_dev(phi)
    g0 = qcd.Gauge.load(to_dev(U), L, BC)
    eta0 = torch.zeros_like(phi_d)
    qcd.solve(g0, f, phi_d, eta0, tol=1e-14, inner="f64", dagger=True)

    def action(Up):
        gp = qcd.Gauge.load(to_dev(Up), L, BC)
        eta = eta0.clone()
        # a fixed number of iterations (tol unreachable), warm-started: identical work for S+ and S-
        info, st = qcd.solve(gp, f, phi_d, eta, tol=1e-30, maxiter=20, inner="f64", dagger=True,
                             x0_given=True, check=False)
        assert st in (qcd.OK, qcd.ERR_NOCONV) and info[0]["true_resid"] < 1e-13
        s = qcd.norm2(gp, f, eta)[0]
        gp.free()
        return s

    rng = np.random.default_rng(1234)
    rms = float(np.sqrt(np.mean(g ** 2)))
    worst = 0.0
    for _ in range(64):
        mu, x, a, b, ri = (int(rng.integers(4)), int(rng.integers(V)), int(rng.integers(3)),
                           int(rng.integers(3)), int(rng.integers(2)))
        d = np.zeros_like(U)
        d[mu, x, a, b] = h * (1.0 if ri == 0 else 1j)
        fd = (action(U + d) - action(U - d)) / (2 * h)
        err = abs(fd - g[mu, x, a, b, ri]) / max(abs(fd), rms)
        worst = max(worst, err)
    print(f"h = {h:g}: S = {S.item():.6e}, worst relative FD deviation {worst:.2e} (rms gradient {rms:.3e})")
    assert worst < FD_TOL[h]
